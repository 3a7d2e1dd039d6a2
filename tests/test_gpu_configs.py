"""Parity of the GPU path with the oracle on the workloads themselves and on
the product paths that only large sizes reach, through the C-ABI.

* the dense 2-D workload (n = 1,000, exponential kernel, no nugget, its own
  observations and targets) in both precisions against the dense oracle;
* the PCG product W^T C~_W W v at n = 16,384 (more columns than one work item
  of either FP32 product covers, a ragged last row block) element by element
  against the oracle's P (C + eta I) P v, P = I - X (X^T X)^-1 X^T the
  projector W^T W, formed with the oracle's kernel sums (no dense matrix);
* the symmetric packed product (mixed path, complete pattern) against the
  oracle on small ragged sizes, and the FP32 row panels of a truncated
  pattern against the FP64 product of the same pattern above the panels'
  column-segment width;
* the high-dimensional regime (d = 10, leaf 128, p = 66, matrix-free
  three-step product with its autotuned kernel sum) at n = 32,768: mixed
  against FP64 predictions and the saddle-point residual of both solves,
  evaluated with the oracle's own arithmetic.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import dense, design, matern, mlblup

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import paper_1701_00285_gb300 as pkg
    pkg.lib()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def projected_cov(P, v):
    """Oracle: P (C + eta I) P v with P = I - X (X^T X)^-1 X^T (W^T W)."""
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, P.w, lo, hi)

    def proj(u):
        return u - X @ np.linalg.solve(X.T @ X, X.T @ u)
    return proj(mlblup.cov_matvec(P.points, proj(v), P.nu, P.rho, P.nugget))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", MIXED_TOL)])
def test_dense_2d_workload_matches_dense_oracle(pkg, prec, tol):
    P = wl.dense_2d()
    ref = dense.dense_blup(P.points, P.Z, P.targets, P.w, P.nu, P.rho, P.nugget)
    ctx = pkg.Context(prec, leaf_size=P.leaf_size, pcg_rtol=1e-13 if prec == "fp64" else 1e-10,
                      pcg_maxit=50000)
    ctx.build_basis(P.points, P.w)
    ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)
    beta, info = ctx.solve(P.Z)
    yhat = ctx.predict(P.targets)
    assert info["converged"]
    assert info["symmetric"] == (1 if prec == "mixed" else 0)
    assert rel(yhat, ref["yhat"]) < tol
    # zero nugget: the BLUP interpolates the data (Sec. 5.2, exact at tau = inf)
    at_data = ctx.predict(P.points[:64])
    assert np.abs(at_data - P.Z[:64]).max() < 1e3 * tol * np.abs(P.Z).max()
    ctx.close()


@pytest.fixture(scope="module")
def mid_problem():
    return wl.heldout_5d(N=16384, M=64)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_cw_product_large_matches_oracle_elementwise(pkg, mid_problem, prec, tol):
    P = mid_problem
    ctx = pkg.Context(prec, leaf_size=P.leaf_size)
    ctx.build_basis(P.points, P.w)
    ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
    assert ctx.nwav % 128 != 0               # ragged last row block of the symmetric storage
    v = np.random.default_rng(21).standard_normal(P.N)
    ref = projected_cov(P, v)
    scale = np.abs(ref).max()
    for variant in ((0, 1) if prec == "mixed" else (None,)):
        if variant is not None:
            ctx.set_product_variant(variant)
        got = ctx.apply_Wt(ctx.cw_matvec(ctx.apply_W(v)))
        assert np.abs(got - ref).max() < tol * scale
        assert rel(got, ref) < tol
    ctx.close()


@pytest.mark.parametrize("seed,N,d,w,n0", [(31, 700, 2, 1, 32), (32, 1000, 3, 1, 64), (33, 2200, 5, 1, 64),
                                            (34, 200, 2, 2, 16)])
def test_symmetric_product_matches_oracle(pkg, seed, N, d, w, n0):
    """Sizes around the 128-row blocks: fewer rows than one block, a few blocks
    with a ragged last one, and the diagonal squares of every block."""
    P = wl.small_problem(seed, N, d, w, nu=1.5, rho=0.3, nugget=1e-4, leaf_size=n0)
    ctx = pkg.Context("mixed", leaf_size=n0)
    ctx.build_basis(P.points, w)
    ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
    rng = np.random.default_rng(seed)
    for _ in range(2):
        v = rng.standard_normal(P.N)
        got = ctx.apply_Wt(ctx.cw_matvec(ctx.apply_W(v)))
        ref = projected_cov(P, v)
        assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max()
    # the same product twice gives the same bits (fixed summation order); the
    # two forms (plain loads, bulk-copy pipeline) agree to FP32 rounding
    u = rng.standard_normal(ctx.nwav)
    outs = []
    for v in (0, 1):
        ctx.set_product_variant(v)
        outs.append(ctx.cw_matvec(u))
        assert np.array_equal(outs[-1], ctx.cw_matvec(u))
    assert np.abs(outs[0] - outs[1]).max() <= 1e-6 * np.abs(outs[0]).max()
    ctx.close()


def test_truncated_fp32_panels_match_fp64_above_segment_width(pkg):
    """A truncated pattern keeps the FP32 row panels (both triangles); at
    n = 16,384 and tau = 0.5 level-mean diameters the leaf panels hold 9,406 to
    16,378 columns, more than one column segment, so the product sums several
    segment partials per row."""
    P = wl.heldout_5d(N=16384, M=64)
    out = {}
    for prec in ("fp64", "mixed"):
        ctx = pkg.Context(prec, leaf_size=P.leaf_size)
        ctx.build_basis(P.points, P.w)
        ctx.assemble(P.nu, P.rho, P.nugget, 0.5)
        info = ctx.info()
        u = np.random.default_rng(22).standard_normal(ctx.nwav)
        out[prec] = (ctx.cw_matvec(u), info)
        ctx.close()
    assert out["mixed"][1]["symmetric"] == 0
    assert out["mixed"][1]["col_total"] > 0
    assert out["mixed"][1]["nnz"] < out["mixed"][1]["product_values"] + 1   # both triangles streamed
    assert rel(out["mixed"][0], out["fp64"][0]) < 1e-6


def test_high_dimension_regime_n32768(pkg):
    """d = 10, leaf 128, w = 2 (p = 66), matrix-free three-step product, the
    regime of the high-dimensional workload at n = 32,768."""
    P = wl.uniform_10d(N=32768, M=1024)
    out = {}
    for prec in ("mixed", "fp64"):
        ctx = pkg.Context(prec, leaf_size=P.leaf_size, pcg_rtol=P.pcg_rtol, pcg_maxit=50000, precond=False,
                          matrix_free=True)
        ctx.build_basis(P.points, P.w)
        ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
        beta, info = ctx.solve(P.Z)
        assert info["converged"], prec
        out[prec] = {"beta": beta, "gamma": ctx.gamma(), "yhat": ctx.predict(P.targets)}
        ctx.close()
    assert rel(out["mixed"]["yhat"], out["fp64"]["yhat"]) < MIXED_TOL
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, P.w, lo, hi)
    for prec, res_tol in (("fp64", 1e-6), ("mixed", 1e-5)):
        g, b = out[prec]["gamma"], out[prec]["beta"]
        r = P.Z - mlblup.cov_matvec(P.points, g, P.nu, P.rho, P.nugget) - X @ b
        assert np.linalg.norm(r) / np.linalg.norm(P.Z) < res_tol, prec
        assert np.linalg.norm(X.T @ g) <= 1e-9 * np.linalg.norm(X) * np.linalg.norm(g)
    # predictions are k(x0)^T beta + c(x0)^T gamma, recomputed by the oracle at 64 targets
    tg = P.targets[:64]
    ref = (design.design_matrix(tg, P.w, lo, hi) @ out["fp64"]["beta"]
           + matern.kernel_matvec(tg, P.points, out["fp64"]["gamma"], P.nu, P.rho))
    assert rel(out["fp64"]["yhat"][:64], ref) < 1e-10


@pytest.mark.parametrize("d", [10, 5])
def test_tensor_core_kernel_sum_matches_fp64(pkg, d):
    """The matrix-free product with its kernel sum on the tensor cores (squared
    distances as one BF16x3 contraction, variant 6) against the FP64 product
    and the FP32 CUDA-core form, on a ragged size (4,000 points: a partial last
    target block and source tile) with the sources split over CTAs."""
    P = wl.uniform_10d(N=4000, M=16) if d == 10 else wl.heldout_5d(N=4000, M=16)
    leaf = 128 if d == 10 else 64
    ref = pkg.Context("fp64", leaf_size=leaf, matrix_free=True, precond=False)
    ref.build_basis(P.points, P.w)
    ref.assemble(P.nu, P.rho, P.nugget, math.inf)
    u = np.random.default_rng(31).standard_normal(ref.nwav)
    want = ref.cw_matvec(u)
    ref.close()
    ctx = pkg.Context("mixed", leaf_size=leaf, matrix_free=True, precond=False)
    ctx.build_basis(P.points, P.w)
    ctx.assemble(P.nu, P.rho, P.nugget, math.inf)
    errs = {}
    for v in (1, 6):
        ctx.set_product_variant(v)
        assert ctx.info()["product_variant"] == v
        got = ctx.cw_matvec(u)
        assert np.all(np.isfinite(got))
        errs[v] = rel(got, want)
    ctx.close()
    assert errs[1] < 1e-5
    assert errs[6] < 1e-5, errs


def test_tensor_core_product_blup_matches_dense_oracle(pkg):
    """A mixed matrix-free BLUP whose every product runs on the tensor cores,
    against the dense oracle (the mixed path's 1e-5)."""
    P = wl.small_problem(650, 2000, 10, 1, nu=2.5, rho=0.8, nugget=1e-4, leaf_size=128, M=100)
    ref = dense.dense_blup(P.points, P.Z, P.targets, 1, 2.5, 0.8, 1e-4)
    ctx = pkg.Context("mixed", leaf_size=128, pcg_rtol=1e-12, pcg_maxit=50000, precond=False, matrix_free=True)
    ctx.build_basis(P.points, 1)
    ctx.assemble(2.5, 0.8, 1e-4, math.inf)
    ctx.set_product_variant(6)
    ctx.solve(P.Z)
    got = ctx.predict(P.targets)
    ctx.close()
    assert rel(got, ref["yhat"]) < MIXED_TOL
