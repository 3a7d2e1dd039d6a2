"""Parity of the GPU path (through the C-ABI) with the CPU oracle.

Quantities compared are the ones the method fixes uniquely: the kd-tree
permutation and the block pattern (bit-exact), W^T W (the projector onto the
complement of the trend space), W^T C~_W W v (independent of the orthonormal
basis chosen inside each cell), gamma-hat, beta-hat and the predictions.
Tolerances: FP64 path 1e-9 relative on predictions (1e-12 on the operators),
PCG run to 1e-13 on both sides.
"""
import dataclasses
import math

import numpy as np
import pytest

import workloads as wl
from oracle import assemble as oa, dense, design, matern, mlblup, pattern as op, tree as ot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1701_00285_gb300 as pkg
    pkg.lib()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ctx_for(pkg, P, precision="fp64", rtol=1e-13, **kw):
    ctx = pkg.Context(precision, leaf_size=P.leaf_size, pcg_rtol=rtol, **kw)
    ctx.build_basis(P.points, P.w)
    return ctx


TREE_CASES = [(1000, 2, 1, 64), (777, 3, 2, 16), (64, 2, 1, 64), (65, 2, 1, 64), (1031, 5, 1, 32), (300, 1, 2, 8)]


@pytest.mark.parametrize("N,d,w,n0", TREE_CASES)
def test_tree_permutation_bit_exact(pkg, N, d, w, n0):
    P = wl.small_problem(100 + N, N, d, w, leaf_size=n0, clustered=(d == 3))
    ctx = ctx_for(pkg, P)
    T = ot.build_tree(P.points, n0)
    assert ctx.t == T.t
    assert np.array_equal(ctx.perm(), T.perm)


@pytest.mark.parametrize("N,d,w,n0", [(600, 2, 1, 32), (777, 3, 2, 16), (513, 5, 1, 20), (300, 1, 3, 8)])
def test_basis_operators(pkg, N, d, w, n0):
    P = wl.small_problem(200 + N, N, d, w, leaf_size=n0)
    ctx = ctx_for(pkg, P)
    p = math.comb(d + w, w)
    assert ctx.p == p and ctx.nwav == N - p
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, w, lo, hi)
    for j in range(p):                                   # W X = 0
        assert np.abs(ctx.apply_W(X[:, j])).max() < 1e-12 * np.abs(X[:, j]).max() * math.sqrt(N)
    u = np.random.default_rng(0).standard_normal(N - p)  # W W^T = I
    np.testing.assert_allclose(ctx.apply_W(ctx.apply_Wt(u)), u, atol=1e-12)
    v = np.random.default_rng(1).standard_normal(N)      # W^T W = I - X (X^T X)^-1 X^T
    proj = v - X @ np.linalg.solve(X.T @ X, X.T @ v)
    np.testing.assert_allclose(ctx.apply_Wt(ctx.apply_W(v)), proj, atol=1e-11)


@pytest.mark.parametrize("c", [0.0, 0.5, 2.0, math.inf])
def test_pattern_bit_exact(pkg, c):
    P = wl.small_problem(300, 900, 3, 1, leaf_size=16, clustered=True)
    ctx = ctx_for(pkg, P)
    ctx.assemble(1.5, 0.2, 1e-6, c)
    T = ot.build_tree(P.points, 16)
    for i in range(T.t + 1):
        for j in range(i, T.t + 1):
            ref = op.level_pair_bruteforce(T, i, j, c)
            assert np.array_equal(ctx.pattern(i, j), ref), (i, j)
            assert np.array_equal(ctx.pattern(j, i), ref.T), (j, i)


@pytest.mark.parametrize("c", [math.inf, 2.0, 0.7])
@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_cw_operator_matches_oracle(pkg, c, nu):
    """W^T C~_W W v on both sides (basis-independent)."""
    P = wl.small_problem(310, 700, 2, 2, nu=nu, leaf_size=24, clustered=True)
    ctx = ctx_for(pkg, P)
    ctx.assemble(nu, 0.25, 1e-5, c)
    B = mlblup.setup(P.points, 2, 24)
    A = oa.to_sparse(B, oa.assemble(B, P.points, nu, 0.25, 1e-5, c))
    v = np.random.default_rng(2).standard_normal(P.N)
    ref = B.apply_Wt(A @ B.apply_W(v))
    got = ctx.apply_Wt(ctx.cw_matvec(ctx.apply_W(v)))
    assert rel(got, ref) < 1e-12


def test_kernel_sum_matches_oracle(pkg):
    P = wl.small_problem(320, 1500, 3, 1, leaf_size=32)
    ctx = ctx_for(pkg, P)
    ctx.assemble(2.5, 0.3, 0.0, math.inf)
    a = np.random.default_rng(3).standard_normal(P.N)
    got = ctx.kernel_sum(P.targets, a)
    ref = matern.kernel_matvec(P.targets, P.points, a, 2.5, 0.3)
    assert rel(got, ref) < 1e-13


BLUP_CASES = [  # seed, N, d, w, nu, rho, nugget, n0
    (400, 1000, 2, 1, 0.5, 0.25, 0.0, 64),    # config-1 shape
    (401, 1100, 3, 2, 1.5, 0.2, 1e-6, 32),
    (402, 900, 5, 1, 2.5, 0.5, 1e-5, 40),
    (403, 517, 2, 2, 1.5, 0.3, 1e-4, 16),
]


@pytest.mark.parametrize("seed,N,d,w,nu,rho,nug,n0", BLUP_CASES)
def test_blup_tau_inf_matches_dense_oracle(pkg, seed, N, d, w, nu, rho, nug, n0):
    P = wl.small_problem(seed, N, d, w, nu=nu, rho=rho, nugget=nug, leaf_size=n0, M=200,
                         clustered=(seed % 2 == 1))
    ref = dense.dense_blup(P.points, P.Z, P.targets, w, nu, rho, nug)
    ctx = ctx_for(pkg, P, pcg_maxit=50000)
    ctx.assemble(nu, rho, nug, math.inf)
    beta, info = ctx.solve(P.Z)
    yhat = ctx.predict(P.targets)
    assert info["converged"]
    assert rel(yhat, ref["yhat"]) < 1e-9
    assert rel(beta, ref["beta"]) < 1e-8
    g = ctx.gamma()
    assert rel(g, ref["gamma"]) < 1e-7
    assert np.abs(ref["X"].T @ g).max() < 1e-10 * np.abs(g).sum()   # X^T gamma = 0


@pytest.mark.parametrize("c", [2.0, 1.0])
def test_blup_finite_tau_matches_multilevel_oracle(pkg, c):
    P = wl.small_problem(410, 1200, 3, 2, nu=1.5, rho=0.2, nugget=1e-6, leaf_size=32, clustered=True, M=100)
    ctx = ctx_for(pkg, P, pcg_maxit=50000)
    ctx.assemble(1.5, 0.2, 1e-6, c)
    beta, info = ctx.solve(P.Z)
    yhat = ctx.predict(P.targets)
    B = mlblup.setup(P.points, 2, 32)
    g, b, oi = mlblup.solve(B, P.points, P.Z, 1.5, 0.2, 1e-6, c, exact=True)
    yref = mlblup.predict(B, P.points, g, b, P.targets, 1.5, 0.2)
    assert info["nnz"] == oi["nnz"]
    assert rel(yhat, yref) < 1e-9
    assert rel(beta, b) < 1e-8


def test_polynomial_data_gives_zero_gamma(pkg):
    P = wl.small_problem(420, 800, 3, 2, nu=2.5, rho=0.3, nugget=1e-6, leaf_size=32)
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, 2, lo, hi)
    beta = np.random.default_rng(4).standard_normal(X.shape[1])
    ctx = ctx_for(pkg, P)
    ctx.assemble(2.5, 0.3, 1e-6, 2.0)
    b, info = ctx.solve(X @ beta)
    np.testing.assert_allclose(b, beta, rtol=1e-10, atol=1e-10)
    assert np.abs(ctx.gamma()).max() < 1e-10


def test_degenerate_single_leaf_and_tiny_p(pkg):
    # N <= n0: the root is the only cell (t = 0); w = 0: constant trend, p = 1
    P = wl.small_problem(430, 50, 2, 0, nu=0.5, rho=0.3, nugget=1e-3, leaf_size=64, M=20)
    ref = dense.dense_blup(P.points, P.Z, P.targets, 0, 0.5, 0.3, 1e-3)
    ctx = ctx_for(pkg, P)
    assert ctx.t == 0 and ctx.p == 1
    ctx.assemble(0.5, 0.3, 1e-3, math.inf)
    ctx.solve(P.Z)
    assert rel(ctx.predict(P.targets), ref["yhat"]) < 1e-10


def test_call_order_and_argument_errors(pkg):
    ctx = pkg.Context("fp64", leaf_size=16)
    with pytest.raises(pkg.MLBError) as e:
        ctx.assemble(1.5, 0.3, 0.0)
    assert e.value.name == "ESTATE"
    P = wl.small_problem(440, 200, 2, 1, leaf_size=16)
    ctx.build_basis(P.points, 1)
    with pytest.raises(pkg.MLBError) as e:
        ctx.solve(P.Z)
    assert e.value.name == "ESTATE"
    with pytest.raises(pkg.MLBError) as e:
        ctx.assemble(0.1, 0.3, 0.0)          # smoothness below the supported range
    assert e.value.name == "EINVAL"
    with pytest.raises(pkg.MLBError) as e:
        ctx.assemble(1.5, 0.3, 0.0, axis=[1.0, -2.0])
    assert e.value.name == "EINVAL"
    with pytest.raises(pkg.MLBError) as e:
        ctx.assemble(1.5, 0.3, 0.0, axis=[1.0, 2.0, 3.0])   # d = 2
    assert e.value.name == "EINVAL"
    with pytest.raises(pkg.MLBError) as e:
        ctx.assemble(1.5, -1.0, 0.0)
    assert e.value.name == "EINVAL"
    bad = P.points.copy()
    bad[3, 0] = np.nan
    with pytest.raises(pkg.MLBError) as e:
        ctx.build_basis(bad, 1)
    assert e.value.name == "EINVAL"
    big = pkg.Context("fp64", leaf_size=128)
    big.build_basis(wl.small_problem(441, 600, 2, 1).points, 1)
    with pytest.raises(pkg.MLBError) as e:
        big.assemble(1.5, 0.3, 0.0)
    assert e.value.name == "EINVAL"
    line = np.zeros((100, 2))
    line[:, 0] = np.linspace(0, 1, 100)
    with pytest.raises(pkg.MLBError) as e:
        pkg.Context("fp64", leaf_size=16).build_basis(line, 1)
    assert e.value.name == "ERANK"


def test_pcg_iteration_cap_reports_noconv(pkg):
    P = wl.small_problem(450, 600, 2, 1, nu=1.5, rho=0.3, nugget=1e-8, leaf_size=32)
    ctx = pkg.Context("fp64", leaf_size=32, pcg_rtol=1e-14, pcg_maxit=3)
    ctx.build_basis(P.points, 1)
    ctx.assemble(1.5, 0.3, 1e-8)
    with pytest.raises(pkg.MLBError) as e:
        ctx.solve(P.Z)
    assert e.value.name == "ENOCONV"
    ctx.predict(P.targets)            # last iterate is still usable


# ---- mixed precision and the matrix-free three-step product ---------------------

MIXED_TOL = 1e-5      # relative prediction error of the mixed path (FP32 tiles)


@pytest.mark.parametrize("seed,N,d,w,nu,rho,nug,n0", [
    (500, 2000, 5, 1, 1.5, 0.3, 1e-4, 64),      # config-5 shape
    (501, 1500, 3, 1, 2.5, 0.4, 1e-4, 32),
    (502, 1200, 2, 1, 0.5, 0.25, 1e-4, 64),
])
def test_mixed_assembled_matches_fp64(pkg, seed, N, d, w, nu, rho, nug, n0):
    P = wl.small_problem(seed, N, d, w, nu=nu, rho=rho, nugget=nug, leaf_size=n0, M=300)
    out = {}
    for prec in ("fp64", "mixed"):
        ctx = ctx_for(pkg, P, prec, rtol=1e-10, pcg_maxit=50000)
        ctx.assemble(nu, rho, nug, math.inf)
        b, info = ctx.solve(P.Z)
        out[prec] = (ctx.predict(P.targets), b, info)
    ref = dense.dense_blup(P.points, P.Z, P.targets, w, nu, rho, nug)
    assert rel(out["fp64"][0], ref["yhat"]) < 1e-9
    assert rel(out["mixed"][0], out["fp64"][0]) < MIXED_TOL
    assert rel(out["mixed"][0], ref["yhat"]) < MIXED_TOL


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", MIXED_TOL)])
def test_matrix_free_matches_dense_oracle(pkg, prec, tol):
    P = wl.small_problem(510, 1500, 4, 2, nu=2.5, rho=0.5, nugget=1e-5, leaf_size=40, M=200)
    ctx = pkg.Context(prec, leaf_size=40, pcg_rtol=1e-12, pcg_maxit=50000, precond=False, matrix_free=True)
    ctx.build_basis(P.points, 2)
    ctx.assemble(2.5, 0.5, 1e-5, math.inf)
    b, info = ctx.solve(P.Z)
    ref = dense.dense_blup(P.points, P.Z, P.targets, 2, 2.5, 0.5, 1e-5)
    assert rel(ctx.predict(P.targets), ref["yhat"]) < tol
    assert rel(b, ref["beta"]) < 100 * tol


def test_matrix_free_product_equals_assembled(pkg):
    P = wl.small_problem(520, 900, 3, 1, leaf_size=32)
    a = ctx_for(pkg, P)
    a.assemble(1.5, 0.3, 1e-3, math.inf)
    m = pkg.Context("fp64", leaf_size=32, matrix_free=True)
    m.build_basis(P.points, 1)
    m.assemble(1.5, 0.3, 1e-3, math.inf)
    u = np.random.default_rng(5).standard_normal(a.nwav)
    assert rel(m.cw_matvec(u), a.cw_matvec(u)) < 1e-12
    with pytest.raises(pkg.MLBError):
        m.assemble(1.5, 0.3, 1e-3, 2.0)           # the three-step product has no truncation


def test_large_leaf_high_dimension_basis(pkg):
    """Leaf size 128 and p = 66 (d = 10, w = 2): the basis of the high-dimensional
    matrix-free workload, checked through its operators."""
    P = wl.small_problem(530, 1100, 10, 2, leaf_size=128)
    ctx = ctx_for(pkg, P)
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, 2, lo, hi)
    v = np.random.default_rng(6).standard_normal(P.N)
    proj = v - X @ np.linalg.solve(X.T @ X, X.T @ v)
    np.testing.assert_allclose(ctx.apply_Wt(ctx.apply_W(v)), proj, atol=1e-10)


# ---- gradient of the held-out loss ----------------------------------------------

def test_grad_matches_dense_oracle_gradient(pkg):
    """n = 2,000 subsample of the differentiation workload, FP64 path vs the
    oracle's dense adjoint gradient."""
    from oracle import grad as og
    P = wl.subsample(wl.heldout_5d(N=8192, M=1024), 2000, seed=3, m=300)
    ctx = ctx_for(pkg, P, rtol=1e-12, pcg_maxit=50000)
    ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
    ctx.solve(P.Z)
    got = ctx.grad(P.targets, P.y_targets)
    ref = og.grad_dense(P.points, P.Z, P.targets, P.y_targets, P.w, P.nu, P.rho, P.nugget)
    np.testing.assert_allclose(got, ref, rtol=1e-7)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grad_matches_central_difference(pkg, prec):
    """Central differences (h = 1e-4) of the library's own loss.  On the FP64
    path d/dlog(rho) agrees to 1e-6 and the small d/dlog(nugget) to the noise of
    a difference quotient of a loss solved to 1e-12.  On the mixed path the loss carries
    ~1e-7 relative noise, i.e. ~loss * 1e-7 / (2h) in a difference quotient, so
    d/dlog(rho) is checked to 1e-3 and the (small) d/dlog(nugget) to that noise
    level; the mixed adjoint gradient must also match the FP64 one to 1e-4."""
    P = wl.small_problem(540, 1200, 5, 1, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=64, M=200, with_y=True)
    ctx = ctx_for(pkg, P, prec, rtol=1e-12, pcg_maxit=50000)

    def loss(rho, nug):
        ctx.assemble(1.5, rho, nug, math.inf)
        ctx.solve(P.Z)
        y = ctx.predict(P.targets)
        return float(np.mean((y - P.y_targets) ** 2))

    h = 1e-4
    fd_rho = (loss(0.3 * math.exp(h), 1e-4) - loss(0.3 * math.exp(-h), 1e-4)) / (2 * h)
    fd_nug = (loss(0.3, 1e-4 * math.exp(h)) - loss(0.3, 1e-4 * math.exp(-h))) / (2 * h)
    ctx.assemble(1.5, 0.3, 1e-4, math.inf)
    ctx.solve(P.Z)
    L, g_rho, g_nug = ctx.grad(P.targets, P.y_targets)
    assert abs(L - loss(0.3, 1e-4)) < 1e-12 + 1e-9 * abs(L)
    if prec == "fp64":
        # PCG to 1e-12 leaves ~1e-10 relative noise in the loss: ~L 5e-7 in a quotient
        assert abs(g_rho - fd_rho) <= 1e-6 * abs(fd_rho)
        assert abs(g_nug - fd_nug) <= max(1e-6 * abs(fd_nug), L * 1e-9 / (2 * h))
    else:
        noise = L * 1e-6 / (2 * h)
        assert abs(g_rho - fd_rho) <= 1e-3 * abs(fd_rho)
        assert abs(g_nug - fd_nug) <= noise
        ref = ctx_for(pkg, P, "fp64", rtol=1e-12, pcg_maxit=50000)
        ref.assemble(1.5, 0.3, 1e-4, math.inf)
        ref.solve(P.Z)
        _, r_rho, r_nug = ref.grad(P.targets, P.y_targets)
        assert abs(g_rho - r_rho) <= 1e-4 * abs(r_rho)
        assert abs(g_nug - r_nug) <= 1e-4 * abs(r_nug)


def test_grad_through_torch_autograd(pkg):
    import torch
    from paper_1701_00285_gb300.autograd import held_out_loss
    P = wl.small_problem(541, 900, 3, 1, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=32, M=100, with_y=True)
    ctx = ctx_for(pkg, P, rtol=1e-12)
    prob = {"context": ctx, "nu": 1.5, "Z": P.Z, "targets": P.targets, "y": P.y_targets}
    lr = torch.tensor(math.log(0.3), dtype=torch.float64, requires_grad=True)
    ln = torch.tensor(math.log(1e-4), dtype=torch.float64, requires_grad=True)
    out = held_out_loss(lr, ln, prob)
    out.backward()
    L, g1, g2 = ctx.grad(P.targets, P.y_targets)
    assert abs(float(out) - L) < 1e-14 and abs(float(lr.grad) - g1) < 1e-14 and abs(float(ln.grad) - g2) < 1e-14


# ---- the configurations' own regimes ---------------------------------------------

def test_high_dimension_subsample_matrix_free(pkg):
    """2,048-point subsample of the d = 10 workload (nu = 5/2, rho = 0.5,
    nugget 1e-5, w = 2, leaf 128): FP64 and mixed three-step PCG vs the dense
    oracle."""
    P = wl.subsample(wl.uniform_10d(N=16384, M=512), 2048, seed=2, m=256)
    ref = dense.dense_blup(P.points, P.Z, P.targets, P.w, P.nu, P.rho, P.nugget)
    got = {}
    for prec in ("fp64", "mixed"):
        ctx = pkg.Context(prec, leaf_size=128, pcg_rtol=1e-12, pcg_maxit=20000, precond=False, matrix_free=True)
        ctx.build_basis(P.points, P.w)
        ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
        ctx.solve(P.Z)
        got[prec] = ctx.predict(P.targets)
    assert rel(got["fp64"], ref["yhat"]) < 1e-9
    assert rel(got["mixed"], ref["yhat"]) < MIXED_TOL


def test_batched_problems_mixed_vs_oracle(pkg):
    """Problems drawn from the batched workload's generator (d in {2,3,5}, all
    three nu, rho in [0.1, 0.5]) truncated at tau = 2 diameters, both
    precisions vs the multilevel oracle's exact solve of the same truncated
    system."""
    probs = [dataclasses.replace(q, tau_factor=2.0) for q in wl.batched_problems(count=60) if q.N <= 1400][:4]
    assert len(probs) == 4
    for P in probs:
        B = mlblup.setup(P.points, P.w, P.leaf_size)
        g, b, _ = mlblup.solve(B, P.points, P.Z, P.nu, P.rho, P.nugget, P.tau_factor, exact=True)
        yref = mlblup.predict(B, P.points, g, b, P.targets[:200], P.nu, P.rho)
        for prec, tol in (("fp64", 1e-9), ("mixed", MIXED_TOL)):
            ctx = ctx_for(pkg, P, prec, rtol=1e-12, pcg_maxit=50000)
            ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)
            ctx.solve(P.Z)
            assert rel(ctx.predict(P.targets[:200]), yref) < tol, (P.name, prec)


def test_mixed_one_shot_kernel_sums_are_double_float_accurate(pkg):
    """The mixed path evaluates the trend and prediction kernel sums in
    double-float on the FP32 pipes: they match FP64 to ~1e-12 even with
    oscillating weights (FP32 kernel values would give ~1e-7 and worse)."""
    P = wl.small_problem(560, 1500, 3, 1, nu=2.5, rho=0.4, leaf_size=32, M=200)
    c64, cmx = ctx_for(pkg, P, "fp64"), ctx_for(pkg, P, "mixed")
    for c in (c64, cmx):
        c.assemble(2.5, 0.4, 1e-4, math.inf)
    rng = np.random.default_rng(7)
    a = rng.standard_normal(P.N)
    assert rel(cmx.kernel_sum(P.targets, a), c64.kernel_sum(P.targets, a)) < 1e-11
    osc = a * 1e3 - np.mean(a * 1e3)                   # cancelling weights
    assert rel(cmx.kernel_sum(P.targets, osc), c64.kernel_sum(P.targets, osc)) < 1e-10


# ---- many problems in one call --------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", MIXED_TOL)])
def test_batch_solve_matches_oracle(pkg, prec, tol):
    """Problems of the batched workload's generator (different n, d, nu, rho;
    tau = 2 diameters) through mlb_batch_solve, each against the multilevel
    oracle's exact solve of its own truncated system."""
    from paper_1701_00285_gb300.binding import batch_solve
    probs = [dataclasses.replace(q, tau_factor=2.0) for q in wl.batched_problems(count=80) if q.N <= 1500][:6]
    items = [{"points": q.points, "w": q.w, "nu": q.nu, "rho": q.rho, "nugget": q.nugget,
              "tau_factor": q.tau_factor, "Z": q.Z, "targets": q.targets[:150]} for q in probs]
    res, ms, st = batch_solve(items, precision=prec, pcg_rtol=1e-12, pcg_maxit=50000)
    from paper_1701_00285_gb300 import lib
    assert st == 0 and ms > 0, lib().mlb_batch_last_error().decode()
    for q, (y, b, s, its) in zip(probs, res):
        assert s == 0 and its > 0
        B = mlblup.setup(q.points, q.w, q.leaf_size)
        g, bb, _ = mlblup.solve(B, q.points, q.Z, q.nu, q.rho, q.nugget, q.tau_factor, exact=True)
        yref = mlblup.predict(B, q.points, g, bb, q.targets[:150], q.nu, q.rho)
        assert rel(y, yref) < tol, q.name
        assert rel(b, bb) < 1e3 * tol, q.name


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", MIXED_TOL)])
def test_batch_solve_mixed_sizes_dense_oracle(pkg, prec, tol):
    """A batch of systems of different sizes in the persistent dataflow launch
    (tau = infinity: symmetric chunks in the mixed path, dense row panels in
    FP64); each must equal the dense BLUP of its own data."""
    from paper_1701_00285_gb300.binding import batch_solve
    small = [q for q in wl.batched_problems(count=40) if q.N <= 1000][:2]
    big = wl.small_problem(590, 2600, 3, 1, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=64, M=150)
    probs = small + [big]
    items = [{"points": q.points, "w": q.w, "nu": q.nu, "rho": q.rho, "nugget": q.nugget,
              "tau_factor": math.inf, "Z": q.Z, "targets": q.targets[:150]} for q in probs]
    res, ms, st = batch_solve(items, precision=prec, pcg_rtol=1e-12, pcg_maxit=50000)
    from paper_1701_00285_gb300 import lib
    assert st == 0, lib().mlb_batch_last_error().decode()
    for q, (y, b, s, its) in zip(probs, res):
        assert s == 0 and its > 0, q.name
        ref = dense.dense_blup(q.points, q.Z, q.targets[:150], q.w, q.nu, q.rho, q.nugget)
        assert rel(y, ref["yhat"]) < tol, (q.name, prec)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_batch_solve_wide_system_on_stream_pool(pkg, prec, tol):
    """A system wider than the persistent launch takes (12,288 unknowns) runs
    the single-problem PCG on the stream pool while two small ones run in the
    launch: the wide one must agree with the same problem solved alone."""
    from paper_1701_00285_gb300.binding import batch_solve
    small = [q for q in wl.batched_problems(count=40) if q.N <= 1000][:2]
    wide = wl.small_problem(591, 13000, 3, 1, nu=1.5, rho=0.2, nugget=1e-4, leaf_size=64, M=100)
    probs = small + [wide]
    items = [{"points": q.points, "w": q.w, "nu": q.nu, "rho": q.rho, "nugget": q.nugget,
              "tau_factor": math.inf, "Z": q.Z, "targets": q.targets[:100]} for q in probs]
    res, ms, st = batch_solve(items, precision=prec, pcg_rtol=1e-10, pcg_maxit=50000)
    from paper_1701_00285_gb300 import lib
    assert st == 0, lib().mlb_batch_last_error().decode()
    assert wide.N - (wide.d + 1) > 12288
    ctx = ctx_for(pkg, wide, prec, rtol=1e-10, pcg_maxit=50000)
    ctx.assemble(wide.nu, wide.rho, wide.nugget, math.inf)
    beta, info = ctx.solve(wide.Z)
    yref = ctx.predict(wide.targets[:100])
    y, b, s, its = res[2]
    assert s == 0 and its > 0
    assert rel(y, yref) < tol
    for q, (y, b, s, its) in zip(small, res[:2]):
        ref = dense.dense_blup(q.points, q.Z, q.targets[:100], q.w, q.nu, q.rho, q.nugget)
        assert s == 0 and rel(y, ref["yhat"]) < (1e-8 if prec == "fp64" else MIXED_TOL), q.name


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_solve_edge_cases(pkg, prec):
    """Edge cases of the persistent launch, beside a regular problem:
    - a system of one 128-row block (no column pieces);
    - data in the trend space, so Z_W is zero up to rounding and the
      predictions are the trend alone;
    - a one-leaf problem whose N is one more than p (a single wavelet)."""
    from paper_1701_00285_gb300.binding import batch_solve
    regular = wl.small_problem(592, 1500, 2, 1, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=64, M=40)
    tiny = wl.small_problem(593, 100, 2, 1, nu=0.5, rho=0.2, nugget=1e-4, leaf_size=128, M=40)
    flat = wl.small_problem(594, 700, 3, 1, nu=2.5, rho=0.3, nugget=1e-4, leaf_size=64, M=40)
    lo, hi = design.box(flat.points)
    beta_true = np.random.default_rng(5).standard_normal(4)
    flat_Z = design.design_matrix(flat.points, 1, lo, hi) @ beta_true
    single = wl.small_problem(595, 4, 2, 1, nu=1.5, rho=0.3, nugget=1e-2, leaf_size=64, M=10)
    probs = [regular, tiny, flat, single]
    Zs = [regular.Z, tiny.Z, flat_Z, single.Z]
    items = [{"points": q.points, "w": q.w, "nu": q.nu, "rho": q.rho, "nugget": q.nugget,
              "tau_factor": math.inf, "Z": z, "targets": q.targets} for q, z in zip(probs, Zs)]
    res, ms, st = batch_solve(items, precision=prec, pcg_rtol=1e-12, pcg_maxit=50000)
    from paper_1701_00285_gb300 import lib
    assert st == 0, lib().mlb_batch_last_error().decode()
    tol = 1e-9 if prec == "fp64" else MIXED_TOL
    for q, z, (y, b, s, its) in zip(probs, Zs, res):
        ref = dense.dense_blup(q.points, z, q.targets, q.w, q.nu, q.rho, q.nugget)
        assert s == 0, q.name
        assert rel(y, ref["yhat"]) < tol, (q.name, prec)
    np.testing.assert_allclose(res[2][1], beta_true, rtol=1e-8, atol=1e-8)


# ---- kriging mean squared error ---------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 1e-5)])
def test_mse_matches_dense_oracle(pkg, prec, tol):
    """MSE at targets and at data points (tau = infinity) against the dense
    oracle's formula; absolute error in units of the process variance."""
    P = wl.small_problem(600, 1500, 2, 1, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=32, M=40)
    tg = np.vstack([P.points[:5], P.targets[:35]])
    ref = dense.mse_at(P.points, tg, P.w, P.nu, P.rho, P.nugget)
    ctx = ctx_for(pkg, P, prec, rtol=1e-12, pcg_maxit=50000)
    with pytest.raises(pkg.MLBError):
        ctx.mse(tg)                                     # before mlb_assemble: MLB_ESTATE
    ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
    got = ctx.mse(tg)
    assert np.max(np.abs(got - ref)) < tol
    assert np.all(got[:5] < 1e-3) and np.all(got > -tol)


def test_mse_matrix_free_matches_assembled(pkg):
    """The same MSE through the three-step product (no assembled C~_W)."""
    P = wl.small_problem(601, 900, 3, 1, nu=2.5, rho=0.4, nugget=1e-4, leaf_size=32, M=8)
    got = {}
    for mf in (False, True):
        ctx = pkg.Context("fp64", leaf_size=32, pcg_rtol=1e-12, pcg_maxit=50000, matrix_free=mf, precond=not mf)
        ctx.build_basis(P.points, P.w)
        ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
        got[mf] = ctx.mse(P.targets)
    ref = dense.mse_at(P.points, P.targets, P.w, P.nu, P.rho, P.nugget)
    assert np.max(np.abs(got[False] - ref)) < 1e-8
    assert np.max(np.abs(got[True] - ref)) < 1e-8


# ---- multilevel log-likelihood ------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_loglik_matches_oracle(pkg, prec, tol):
    """Quadratic form against the oracle's exact solve; the stochastic Lanczos
    log-determinant against the oracle's estimate with the same probes and
    steps (the same recurrence, rotated within each cell's wavelet block);
    and the likelihood formula."""
    from oracle import loglik as olog
    P = wl.small_problem(610, 700, 2, 1, nu=1.5, rho=0.3, nugget=1e-3, leaf_size=32, M=8)
    B = mlblup.setup(P.points, P.w, P.leaf_size)
    probes = np.random.default_rng(5).choice([-1.0, 1.0], size=(6, P.N))
    _, ld_ref, q_ref = olog.multilevel_loglik(B, P.points, P.Z, P.nu, P.rho, P.nugget, probes=probes, steps=20)
    ctx = ctx_for(pkg, P, prec, rtol=1e-12, pcg_maxit=50000)
    ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
    l, ld, q = ctx.loglik(P.Z, probes, 20)
    assert abs(q - q_ref) < tol * abs(q_ref)
    assert abs(ld - ld_ref) < tol * max(1.0, abs(ld_ref))
    n = P.N - B.p
    assert abs(l + 0.5 * (n * math.log(2 * math.pi) + ld + q)) < 1e-12 * abs(l)
    l0, ld0, q0 = ctx.loglik(P.Z)                       # no probes: no estimate
    assert ld0 == 0.0 and abs(q0 - q) < 1e-9 * abs(q)
