"""Pins of the BLUP solvers: dense (eqs. GLSbeta, KrigBLUP, Spatial:problem)
and multilevel (eqs. Spatial:eqn1-3), against properties the paper and the
mathematics fix."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import assemble as oa, dense, design, matern, mlblup, pcg as opcg


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_exact_interpolation_without_nugget():
    P = wl.small_problem(10, 150, 2, 1, nu=1.5, rho=0.2, nugget=0.0)
    r = dense.dense_blup(P.points, P.Z, P.points[:20], P.w, P.nu, P.rho, 0.0)
    np.testing.assert_allclose(r["yhat"], P.Z[:20], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("path", ["dense", "multilevel"])
def test_polynomial_data_recovers_coefficients(path):
    P = wl.small_problem(11, 200, 3, 2, nu=2.5, rho=0.3, nugget=1e-6, leaf_size=16)
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, 2, lo, hi)
    beta = np.random.default_rng(0).standard_normal(X.shape[1])
    Z = X @ beta
    if path == "dense":
        r = dense.dense_blup(P.points, Z, P.targets, 2, P.nu, P.rho, P.nugget)
    else:
        r = mlblup.blup(P.points, Z, P.targets, 2, P.nu, P.rho, P.nugget, 16, exact=True)
    np.testing.assert_allclose(r["beta"], beta, rtol=1e-9, atol=1e-9)
    assert np.abs(r["gamma"]).max() < 1e-8


def test_gls_equals_saddle_point_and_constraint():
    P = wl.small_problem(12, 180, 2, 2, nu=0.5, rho=0.3, nugget=1e-4)
    r = dense.dense_blup(P.points, P.Z, P.targets, P.w, P.nu, P.rho, P.nugget)
    g, b = dense.saddle_point_solve(P.points, P.Z, P.w, P.nu, P.rho, P.nugget)
    np.testing.assert_allclose(r["beta"], b, rtol=1e-9)
    np.testing.assert_allclose(r["gamma"], g, rtol=1e-8, atol=1e-10)
    assert np.abs(r["X"].T @ r["gamma"]).max() < 1e-9 * np.abs(r["gamma"]).max() * 180


CASES = [  # seed, N, d, w, nu, rho, nugget, n0
    (20, 300, 2, 1, 0.5, 0.25, 0.0, 16),
    (21, 257, 3, 2, 1.5, 0.2, 1e-6, 16),
    (22, 200, 5, 1, 2.5, 0.5, 1e-5, 12),
    (23, 240, 2, 2, 1.5, 0.3, 1e-4, 8),
]


@pytest.mark.parametrize("seed,N,d,w,nu,rho,nug,n0", CASES)
def test_multilevel_equals_dense_at_tau_inf(seed, N, d, w, nu, rho, nug, n0):
    """Sec. 5.2: the multilevel predictor solves eq. Spatial:problem exactly."""
    P = wl.small_problem(seed, N, d, w, nu=nu, rho=rho, nugget=nug, leaf_size=n0, clustered=(seed % 2 == 1))
    rd = dense.dense_blup(P.points, P.Z, P.targets, w, nu, rho, nug)
    rm = mlblup.blup(P.points, P.Z, P.targets, w, nu, rho, nug, n0, exact=True)
    assert rel(rm["yhat"], rd["yhat"]) < 1e-9
    assert rel(rm["beta"], rd["beta"]) < 1e-8
    rp = mlblup.blup(P.points, P.Z, P.targets, w, nu, rho, nug, n0, rtol=1e-13, maxit=5000)
    assert rp["info"]["converged"]
    assert rel(rp["yhat"], rd["yhat"]) < 1e-8


def test_assembled_equals_three_step_product():
    P = wl.small_problem(24, 200, 3, 1, nugget=1e-3, leaf_size=10)
    B = mlblup.setup(P.points, 1, 10)
    A = oa.to_sparse(B, oa.assemble(B, P.points, P.nu, P.rho, P.nugget, math.inf)).toarray()
    W = B.dense_W()
    C = matern.covariance(P.points, P.nu, P.rho, P.nugget)
    np.testing.assert_allclose(A, W @ C @ W.T, atol=1e-12)
    u = np.random.default_rng(0).random(B.nwav)
    three = B.apply_W(mlblup.cov_matvec(P.points, B.apply_Wt(u), P.nu, P.rho, P.nugget))
    np.testing.assert_allclose(A @ u, three, atol=1e-11)


def test_condition_numbers_props_1_and_2():
    """Prop. 1: kappa(C_W) <= kappa(C); Prop. 2: the upper-left blocks C^n_W
    (finest levels t..n) have non-increasing condition numbers towards n = t;
    Thm. after the P_W remark: diag(C_W) > 0."""
    P = wl.small_problem(25, 256, 2, 2, nu=1.5, rho=0.4, nugget=0.0, leaf_size=16)
    B = mlblup.setup(P.points, 2, 16)
    A = oa.to_sparse(B, oa.assemble(B, P.points, P.nu, P.rho, 0.0, math.inf)).toarray()
    C = matern.covariance(P.points, P.nu, P.rho, 0.0)
    lc = np.linalg.eigvalsh(C)
    la = np.linalg.eigvalsh(A)
    assert la[0] >= lc[0] * (1 - 1e-8) and la[-1] <= lc[-1] * (1 + 1e-12)   # interlacing
    kappas = []
    lev = B.level_of_row()
    for n in range(B.tree.t, -1, -1):
        m = int(np.sum(lev >= n))
        ev = np.linalg.eigvalsh(A[:m, :m])
        kappas.append(ev[-1] / ev[0])
    assert all(k1 <= k2 * (1 + 1e-9) for k1, k2 in zip(kappas, kappas[1:]))
    assert kappas[-1] <= lc[-1] / lc[0]
    assert np.all(np.diag(A) > 0)


def test_nugget_adds_identity_in_wavelet_space():
    P = wl.small_problem(26, 150, 2, 1, leaf_size=10)
    B = mlblup.setup(P.points, 1, 10)
    A0 = oa.to_sparse(B, oa.assemble(B, P.points, 1.5, 0.3, 0.0, math.inf)).toarray()
    A1 = oa.to_sparse(B, oa.assemble(B, P.points, 1.5, 0.3, 0.25, math.inf)).toarray()
    np.testing.assert_allclose(A1 - A0, 0.25 * np.eye(B.nwav), atol=1e-13)


def test_truncation_keeps_pattern_blocks_exactly():
    P = wl.small_problem(27, 300, 2, 1, nugget=1e-4, leaf_size=12, clustered=True)
    B = mlblup.setup(P.points, 1, 12)
    full = oa.to_sparse(B, oa.assemble(B, P.points, 1.5, 0.3, 1e-4, math.inf)).toarray()
    asm = oa.assemble(B, P.points, 1.5, 0.3, 1e-4, 1.0)
    sp = oa.to_sparse(B, asm).toarray()
    mask = sp != 0
    assert 0.05 < mask.mean() < 0.95
    np.testing.assert_allclose(sp[mask], full[mask], atol=1e-14)
    np.testing.assert_allclose(sp, sp.T, atol=0)


def test_pcg_on_known_system_and_unpreconditioned_stop():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    A = Q @ np.diag(np.logspace(0, 4, 60)) @ Q.T
    A = A + np.diag(rng.random(60) * 1e3)
    xs = rng.standard_normal(60)
    b = A @ xs
    res = opcg.pcg(lambda v: A @ v, b, np.diag(A).copy(), 1e-12, 1000)
    assert res.converged and np.linalg.norm(b - A @ res.x) <= 1e-12 * np.linalg.norm(b) * 1.01
    np.testing.assert_allclose(res.x, xs, rtol=1e-6)
    # an indefinite matrix is reported as breakdown
    Ab = np.diag([1.0, -1.0])
    assert opcg.pcg(lambda v: Ab @ v, np.array([0.0, 1.0]), None, 1e-12, 10).breakdown


def test_mse_nonnegative_and_zero_at_data():
    P = wl.small_problem(28, 120, 2, 1, nugget=0.0, leaf_size=10)
    m = dense.mse_at(P.points, np.vstack([P.points[:5], P.targets]), 1, 1.5, 0.3, 0.0)
    assert np.all(m > -1e-8)
    np.testing.assert_allclose(m[:5], 0.0, atol=1e-7)


def test_mse_single_point_closed_form():
    """One observation, constant trend (w = 0), no nugget: the kriging weight
    is forced to 1 by the unbiasedness constraint, so the error variance is
    Var(Z(x0) - Z(x1)) = 2 - 2 phi(|x0 - x1|)."""
    x1 = np.array([[0.3, 0.7]])
    tg = np.array([[0.3, 0.7], [0.5, 0.5], [0.9, 0.1], [3.0, -2.0]])
    for nu in (0.5, 1.5, 2.5):
        m = dense.mse_at(x1, tg, 0, nu, 0.4, 0.0)
        r = np.linalg.norm(tg - x1, axis=1)
        np.testing.assert_allclose(m, 2.0 - 2.0 * matern.matern(r, nu, 0.4), rtol=1e-12, atol=1e-14)


def test_mse_equals_error_variance_of_the_kriging_weights():
    """The MSE formula against its definition: with the weights w0 of the
    predictor Z-hat(x0) = w0^T Z (from the saddle-point system with right-hand
    side [c(x0); k(x0)]), the error variance is phi(0) - 2 w0^T c + w0^T C w0,
    where C carries the nugget and c(x0) does not."""
    P = wl.small_problem(29, 90, 2, 1, nugget=1e-3, leaf_size=10)
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, 1, lo, hi)
    C = matern.covariance(P.points, 1.5, 0.3, 1e-3)
    N, p = X.shape
    K = np.zeros((N + p, N + p))
    K[:N, :N], K[:N, N:], K[N:, :N] = C, X, X.T
    tg = P.targets[:6]
    c0 = matern.kernel_matrix(P.points, tg, 1.5, 0.3)
    k0 = design.design_matrix(tg, 1, lo, hi).T
    w0 = np.linalg.solve(K, np.vstack([c0, k0]))[:N]
    var = 1.0 - 2.0 * np.einsum("ik,ik->k", w0, c0) + np.einsum("ik,ik->k", w0, C @ w0)
    np.testing.assert_allclose(dense.mse_at(P.points, tg, 1, 1.5, 0.3, 1e-3), var, rtol=1e-9, atol=1e-12)
