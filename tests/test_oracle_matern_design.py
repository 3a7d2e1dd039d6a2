"""Pins of the oracle's Matern covariance and design matrix against the
definition (Sec. 3.1), library Bessel functions and the paper's printed p(d, w)."""
import math
import os

import numpy as np
import pytest
from scipy.special import gamma as Gamma, kv

from oracle import design, matern

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "num_monomials.txt")


def matern_definition(r, nu, rho):
    """Def. "Matern covariance function" via scipy's K_nu (limit 1 at r = 0)."""
    s = math.sqrt(2 * nu) * np.asarray(r) / rho
    out = np.ones_like(s)
    nz = s > 0
    out[nz] = s[nz] ** nu * kv(nu, s[nz]) / (Gamma(nu) * 2 ** (nu - 1))
    return out


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
@pytest.mark.parametrize("rho", [0.1, 0.5, 3.0])
def test_closed_form_matches_bessel_definition(nu, rho):
    r = np.concatenate([[0.0], np.logspace(-6, 1.3, 200)])
    np.testing.assert_allclose(matern.matern(r, nu, rho), matern_definition(r, nu, rho),
                               rtol=1e-12, atol=1e-300)


def test_unit_variance_and_monotone():
    for nu in matern.SUPPORTED_NU:
        assert matern.matern(np.array([0.0]), nu, 0.3)[0] == 1.0
        v = matern.matern(np.linspace(0, 5, 500), nu, 0.3)
        assert np.all(np.diff(v) < 0)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_dlogrho_matches_central_difference(nu):
    r = np.linspace(0.0, 2.0, 101)
    rho, h = 0.37, 1e-5
    fd = (matern.matern(r, nu, rho * math.exp(h)) - matern.matern(r, nu, rho * math.exp(-h))) / (2 * h)
    np.testing.assert_allclose(matern.dmatern_dlogrho(r, nu, rho), fd, rtol=1e-8, atol=1e-11)


def test_nonpositive_nu_and_unknown_family_raise():
    with pytest.raises(ValueError):
        matern.matern(np.array([1.0]), -0.5, 1.0)
    with pytest.raises(ValueError):
        matern.matern(np.array([1.0]), 1.5, 1.0, family="cauchy")


GENERAL_NU = [0.3, 0.75, 1.0, 1.25, 3.7]


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_general_nu_path_matches_closed_forms(nu):
    """The K_nu form of the definition (used for every other nu) reproduces the
    half-integer closed forms: pins its constant 1 / (Gamma(nu) 2^(nu-1)) and
    its argument s = sqrt(2 nu) r / rho."""
    r = np.concatenate([[0.0], np.logspace(-5, 1.2, 120)])
    s = math.sqrt(2 * nu) * r / 0.4
    np.testing.assert_allclose(matern.matern_kv(s, nu), matern.matern(r, nu, 0.4), rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(matern.dmatern_kv(s, nu), matern.dmatern_dlogrho(r, nu, 0.4), rtol=1e-11,
                               atol=1e-300)


@pytest.mark.parametrize("nu", GENERAL_NU)
def test_general_nu_matches_integral_representation(nu):
    """K_nu(s) = int_0^inf exp(-s cosh t) cosh(nu t) dt (A&S 9.6.24), by
    adaptive quadrature: independent of the library's K_nu."""
    from scipy.integrate import quad
    for s in (1e-3, 0.05, 0.5, 1.0, 2.0, 5.0, 12.0):
        # past t_max the integrand is below exp(-80) of its peak
        t_max = math.acosh(1.0 + 80.0 / s) + 1.0
        K, _ = quad(lambda t: math.exp(-s * math.cosh(t)) * math.cosh(nu * t), 0.0, t_max,
                    epsabs=0.0, epsrel=1e-13, limit=400)
        ref = s ** nu * K / (Gamma(nu) * 2.0 ** (nu - 1.0))
        got = matern.matern_kv(np.array([s]), nu)[0]
        assert abs(got - ref) <= 1e-10 * abs(ref), (s, got, ref)


@pytest.mark.parametrize("nu", GENERAL_NU)
def test_general_nu_unit_variance_monotone_and_derivative(nu):
    r = np.linspace(0.0, 3.0, 301)
    v = matern.matern(r, nu, 0.5)
    assert v[0] == 1.0 and np.all(np.diff(v) < 0)
    rho, h = 0.37, 1e-5
    r = np.linspace(0.01, 2.0, 60)
    fd = (matern.matern(r, nu, rho * math.exp(h)) - matern.matern(r, nu, rho * math.exp(-h))) / (2 * h)
    np.testing.assert_allclose(matern.dmatern_dlogrho(r, nu, rho), fd, rtol=1e-7, atol=1e-11)


def test_gaussian_is_the_large_nu_limit_of_matern():
    """Remark after the Matern definition: nu -> inf gives exp(-r^2 / (2 rho^2))."""
    r = np.linspace(0.0, 2.0, 81)
    g = matern.matern(r, None, 0.6, family="gaussian")
    errs = [np.abs(matern.matern(r, nu, 0.6) - g).max() for nu in (10.0, 20.0, 60.0)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 4.5e-3
    h = 1e-5
    fd = (matern.matern(r, None, 0.6 * math.exp(h), "gaussian") - matern.matern(r, None, 0.6 * math.exp(-h), "gaussian")) / (2 * h)
    np.testing.assert_allclose(matern.dmatern_dlogrho(r, None, 0.6, "gaussian"), fd, rtol=1e-8, atol=1e-12)


def test_anisotropic_distance_follows_the_definition():
    """r(theta)^2 = (x - y)^T diag(theta) (x - y) (Sec. 3): a hand-worked pair,
    and Euclidean distances of coordinates scaled by sqrt(theta)."""
    x, y = np.array([[1.0, 2.0]]), np.array([[4.0, 6.0]])
    assert matern.distances(x, y, axis=[2.0, 0.5])[0, 0] == math.sqrt(2.0 * 9.0 + 0.5 * 16.0)
    rng = np.random.default_rng(1)
    a, b, th = rng.random((6, 3)), rng.random((4, 3)), np.array([0.3, 2.0, 5.0])
    np.testing.assert_allclose(matern.distances(a, b, th), matern.distances(a * np.sqrt(th), b * np.sqrt(th)),
                               rtol=1e-14)


def test_distances_brute_force():
    rng = np.random.default_rng(0)
    x, y = rng.random((7, 4)), rng.random((5, 4))
    ref = np.array([[math.sqrt(sum((a - b) ** 2 for a, b in zip(xi, yj))) for yj in y] for xi in x])
    np.testing.assert_allclose(matern.distances(x, y), ref, rtol=1e-15)


def test_num_monomials_printed_in_paper():
    rows = [l.split()[:3] for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    assert design.num_monomials(10, 7) != 1001      # the Sec. 8.1 typo (see fixture)
    for d, w, p in rows:
        d, w, p = int(d), int(w), int(p)
        assert design.num_monomials(d, w) == p
        if p <= 1001:
            assert len(design.exponents(d, w)) == p


@pytest.mark.parametrize("d,w", [(1, 3), (2, 2), (3, 2), (5, 1), (10, 2), (4, 3)])
def test_exponents_complete_unique_graded(d, w):
    ex = design.exponents(d, w)
    brute = {a for a in np.ndindex(*([w + 1] * d)) if sum(a) <= w}
    assert set(ex) == brute and len(ex) == len(brute) == math.comb(d + w, w)
    degs = [sum(a) for a in ex]
    assert degs == sorted(degs)
    for deg in range(w + 1):
        block = [a for a in ex if sum(a) == deg]
        assert block == sorted(block, reverse=True)
    assert ex[0] == (0,) * d
    assert ex[1:d + 1] == [tuple(int(i == k) for i in range(d)) for k in range(d)]


def test_design_matrix_columns():
    rng = np.random.default_rng(1)
    x = rng.random((50, 3)) * 4 - 1
    lo, hi = design.box(x)
    X = design.design_matrix(x, 2, lo, hi)
    u = 2 * (x - lo) / (hi - lo) - 1
    assert np.allclose(X[:, 0], 1)
    np.testing.assert_allclose(X[:, 1:4], u, rtol=1e-14)
    np.testing.assert_allclose(X[:, 4], u[:, 0] ** 2, rtol=1e-14)
    np.testing.assert_allclose(X[:, 5], u[:, 0] * u[:, 1], rtol=1e-14)
    assert u.min() == -1.0 and u.max() == 1.0
