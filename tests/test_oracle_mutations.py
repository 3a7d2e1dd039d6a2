"""Planted mistakes: each test injects a plausible bug into the oracle (on the
CPU only) and checks that one of the pins catches it."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import basis as ob, grad, matern, mlblup, pattern as op, tree as ot
from oracle import dense


def test_dropped_term_in_matern_is_caught(monkeypatch):
    from tests.test_oracle_matern_design import matern_definition
    good = matern.matern

    def bad(r, nu, rho):
        if nu == 2.5:
            s = math.sqrt(5.0) * np.asarray(r) / rho
            return (1.0 + s) * np.exp(-s)        # s^2/3 term dropped
        return good(r, nu, rho)

    r = np.linspace(0, 2, 50)
    assert not np.allclose(bad(r, 2.5, 0.4), matern_definition(r, 2.5, 0.4), rtol=1e-6)


def test_wrong_scaling_wavelet_split_is_caught(monkeypatch):
    orig_svd = np.linalg.svd

    def shifted(M, full_matrices=True):
        U, S, Vh = orig_svd(M, full_matrices=full_matrices)
        return U, S, np.roll(Vh, 1, axis=0)      # columns of V out of order
    monkeypatch.setattr(ob.np.linalg, "svd", shifted)
    x = np.random.default_rng(0).random((120, 2))
    try:
        B = ob.build_basis(x, ot.build_tree(x, 10), 1)
    except ob.RankDeficient:
        return
    assert np.abs(B.dense_W() @ B.X).max() > 1e-6


def test_one_sided_box_test_is_caught():
    x = np.array([0.0, 0.1, 0.2, 0.3, 1.0, 1.1, 3.0, 3.1])[:, None]
    T = ot.build_tree(x, 2)
    tau = op.tau_levels(T, 2, 2, 2.0)
    lo_m, hi_m = T.lo[2][:, None, 0], T.hi[2][:, None, 0]
    lo_q, hi_q = T.lo[2][None, :, 0], T.hi[2][None, :, 0]
    bad = ~((lo_q - hi_m) > tau)                 # planted: the lo_m - hi_q side is not tested
    good = op.level_pair_bruteforce(T, 2, 2, 2.0)
    assert not np.array_equal(bad, good)
    assert not np.array_equal(bad, bad.T)        # and the symmetry pin fails too


def test_trend_step_with_wrong_sign_is_caught(monkeypatch):
    P = wl.small_problem(40, 160, 2, 1, nugget=1e-4, leaf_size=12)
    good_cov = mlblup.cov_matvec
    monkeypatch.setattr(mlblup, "cov_matvec", lambda pts, v, nu, rho, nug: -good_cov(pts, v, nu, rho, nug))
    rm = mlblup.blup(P.points, P.Z, P.targets, 1, P.nu, P.rho, P.nugget, 12, exact=True)
    rd = dense.dense_blup(P.points, P.Z, P.targets, 1, P.nu, P.rho, P.nugget)
    assert np.linalg.norm(rm["yhat"] - rd["yhat"]) > 1e-3 * np.linalg.norm(rd["yhat"])


def test_missing_trend_adjoint_is_caught(monkeypatch):
    P = wl.small_problem(41, 160, 2, 1, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=12, with_y=True, M=30)
    d = grad.grad_dense(P.points, P.Z, P.targets, P.y_targets, 1, 1.5, 0.3, 1e-4)
    real_solve = np.linalg.solve
    calls = {"n": 0}

    def zero_lambda0(A, b):
        out = real_solve(A, b)
        if np.ndim(b) == 1 and A.shape == (3, 3):
            calls["n"] += 1
            if calls["n"] == 2:               # the lambda_0 = X (X^T X)^{-1} b solve
                return np.zeros_like(out)
        return out
    monkeypatch.setattr(grad.np.linalg, "solve", zero_lambda0)
    m = grad.grad_multilevel(P.points, P.Z, P.targets, P.y_targets, 1, 1.5, 0.3, 1e-4, 12)
    assert not np.allclose(m[1:], d[1:], rtol=1e-4)


def test_mse_without_the_trend_correction_is_caught():
    """Planted: MSE = 1 - c^T C^{-1} c (simple-kriging variance, the u^T A^{-1} u
    term of the unknown trend dropped).  The one-observation closed form
    2 - 2 phi(r) fails."""
    x1 = np.array([[0.3, 0.7]])
    tg = np.array([[0.5, 0.5], [0.9, 0.1]])
    C = matern.covariance(x1, 1.5, 0.4, 0.0)
    c0 = matern.kernel_matrix(x1, tg, 1.5, 0.4)
    bad = 1.0 - np.einsum("ik,ik->k", c0, np.linalg.solve(C, c0))
    r = np.linalg.norm(tg - x1, axis=1)
    assert not np.allclose(bad, 2.0 - 2.0 * matern.matern(r, 1.5, 0.4), rtol=1e-6)


def test_slq_without_the_probe_norm_is_caught(monkeypatch):
    """Planted: the stochastic Lanczos estimate forgets the |v|^2 factor of
    each probe.  The unit-probe exactness pin fails as soon as the probes are
    not unit vectors, and the Hutchinson bound fails for Rademacher probes."""
    from oracle import loglik
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    A = Q @ np.diag(np.logspace(0.5, 1.5, 60)) @ Q.T
    probes = rng.choice([-1.0, 1.0], size=(200, 60))

    def bad(A, probes, k):
        tot = 0.0
        for v in probes:
            a, b = loglik.lanczos_tridiagonal(A, v, k)
            th, U = np.linalg.eigh(np.diag(a) + np.diag(b, 1) + np.diag(b, -1))
            tot += float(np.sum(U[0] ** 2 * np.log(th)))
        return tot / len(probes)

    exact = np.linalg.slogdet(A)[1]
    lam, U = np.linalg.eigh(A)
    L = (U * np.log(lam)) @ U.T
    sd = math.sqrt(2.0 * (np.sum(L ** 2) - np.sum(np.diag(L) ** 2)) / probes.shape[0])
    assert abs(loglik.slq_logdet(A, probes, 20) - exact) < 4.0 * sd
    assert abs(bad(A, probes, 20) - exact) > 4.0 * sd


def test_loglik_with_the_dense_covariance_is_caught():
    """Planted: the quadratic form taken with C instead of C_W
    (Z^T C^{-1} Z).  The REML quadratic-form pin fails."""
    P = wl.small_problem(31, 140, 2, 1, nu=1.5, rho=0.3, nugget=1e-3, leaf_size=12)
    C = matern.covariance(P.points, P.nu, P.rho, P.nugget)
    from oracle import design as od
    lo, hi = od.box(P.points)
    X = od.design_matrix(P.points, P.w, lo, hi)
    Ci_Z = np.linalg.solve(C, P.Z)
    Ci_X = np.linalg.solve(C, X)
    q_reml = P.Z @ Ci_Z - (X.T @ Ci_Z) @ np.linalg.solve(X.T @ Ci_X, X.T @ Ci_Z)
    bad = float(P.Z @ Ci_Z)
    assert abs(bad - q_reml) > 1e-6 * abs(q_reml)
