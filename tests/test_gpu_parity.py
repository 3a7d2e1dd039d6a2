"""Parity of the GPU path (through the C-ABI) with the CPU oracle.

Quantities compared are the ones the method fixes uniquely: the kd-tree
permutation and the block pattern (bit-exact), W^T W (the projector onto the
complement of the trend space), W^T C~_W W v (independent of the orthonormal
basis chosen inside each cell), gamma-hat, beta-hat and the predictions.
Tolerances: FP64 path 1e-9 relative on predictions (1e-12 on the operators),
PCG run to 1e-13 on both sides.
"""
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
        ctx.assemble(0.75, 0.3, 0.0)
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
