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


def test_unsupported_nu_raises():
    with pytest.raises(ValueError):
        matern.matern(np.array([1.0]), 0.75, 1.0)


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
