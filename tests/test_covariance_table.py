"""The covariance function as the library evaluates it (mlb_covariance: the
host copy of the kernels' FP64 evaluation, no GPU needed) against the
oracle's definition: closed forms, the K_nu form of the definition for any
other smoothness (tabulated in Chebyshev pieces by the library), the Gaussian
kernel and the derivatives in log(rho)."""
import numpy as np
import pytest

from oracle import matern


@pytest.fixture(scope="module")
def cov():
    from paper_1701_00285_gb300 import binding
    binding.lib()
    return binding.covariance


R = np.concatenate([[0.0], np.logspace(-14, 2, 1500)])


@pytest.mark.parametrize("nu,tol", [(0.2, 2e-14), (0.3, 2e-14), (0.75, 2e-14), (1.0, 2e-14), (1.25, 2e-14),
                                    (2.0, 2e-14), (3.7, 5e-14), (12.5, 3e-13), (29.0, 5e-13)])
# (the oracle's own logarithmic evaluation loses about |log phi| + nu ln nu ulps)
def test_tabulated_matern_matches_definition(cov, nu, tol):
    for rho in (0.1, 0.5, 2.0):
        got, ref = cov(R, nu, rho), matern.matern(R, nu, rho)
        assert np.abs(got - ref).max() < tol, (nu, rho)
        gd, rd = cov(R, nu, rho, deriv=True), matern.dmatern_dlogrho(R, nu, rho)
        assert np.abs(gd - rd).max() < 5 * tol, (nu, rho)
    assert cov(np.array([0.0]), nu, 0.5)[0] == 1.0


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_closed_forms_and_gaussian(cov, nu):
    np.testing.assert_allclose(cov(R, nu, 0.4), matern.matern(R, nu, 0.4), rtol=1e-13, atol=1e-30)
    np.testing.assert_allclose(cov(R, nu, 0.4, deriv=True), matern.dmatern_dlogrho(R, nu, 0.4), rtol=1e-13,
                               atol=1e-30)
    g = cov(R, None, 0.7, family="gaussian")
    np.testing.assert_allclose(g, matern.matern(R, None, 0.7, family="gaussian"), rtol=1e-13, atol=1e-30)


def test_table_against_high_precision_bessel(cov):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for nu in (0.3, 0.75, 1.25, 7.3):
        for r in (1e-9, 1e-4, 0.03, 0.4, 1.7, 6.0):
            s = mp.sqrt(2 * nu) * mp.mpf(r) / mp.mpf("0.5")
            exact = s ** nu * mp.besselk(nu, s) / (mp.gamma(nu) * mp.mpf(2) ** (nu - 1))
            assert abs(cov(np.array([r]), nu, 0.5)[0] - float(exact)) < 3e-15, (nu, r)


def test_invalid_parameters_are_rejected(cov):
    from paper_1701_00285_gb300 import MLBError
    for nu, rho in ((0.1, 1.0), (31.0, 1.0), (1.2, 0.0), (1.2, -1.0)):
        with pytest.raises(MLBError):
            cov(np.array([1.0]), nu, rho)
