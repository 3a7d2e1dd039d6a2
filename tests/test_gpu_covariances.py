"""GPU parity for the covariance functions beyond the half-integer Matern
closed forms, through the C-ABI: Matern of any smoothness (the paper's runs
use nu = 3/4 and 5/4, Tables 1-4), the Gaussian kernel of Sec. 8.2 and the
anisotropic distance r(theta) of Sec. 3, against the oracle's definition.

Kernel sums are compared value by value (FP64 path to 1e-13, the mixed
path's double-float sums to 1e-12); predictions at tau = infinity against
the dense oracle (1e-9 FP64, 1e-5 mixed, the tolerances of the half-integer
tests); a finite-tau assembly against the multilevel oracle; the gradient in
log(rho) against the dense oracle's adjoint gradient.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import dense, grad as og, matern, mlblup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1701_00285_gb300 as pkg
    pkg.lib()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


COVS = [  # nu, rho, family, axis
    (0.75, 0.3, "matern", None),
    (1.25, 0.3, "matern", None),
    (1.0, 0.25, "matern", None),
    (0.3, 0.4, "matern", None),
    (3.7, 0.2, "matern", None),
    (None, 0.3, "gaussian", None),
    (1.5, 0.3, "matern", [0.5, 2.0, 8.0]),
    (0.75, 0.3, "matern", [4.0, 1.0, 0.25]),
    (None, 0.5, "gaussian", [1.0, 3.0, 0.5]),
]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 1e-12)])
@pytest.mark.parametrize("nu,rho,family,axis", COVS)
def test_kernel_sum_matches_oracle(pkg, prec, tol, nu, rho, family, axis):
    P = wl.small_problem(600, 1500, 3, 1, leaf_size=32)
    ctx = pkg.Context(prec, leaf_size=32)
    ctx.build_basis(P.points, 1)
    ctx.assemble(nu if nu else 1.5, rho, 0.0, math.inf, family=family, axis=axis)
    a = np.random.default_rng(7).standard_normal(P.N)
    got = ctx.kernel_sum(P.targets, a)
    ref = matern.kernel_matvec(P.targets, P.points, a, nu, rho, family=family, axis=axis)
    ctx.close()
    assert rel(got, ref) < tol


BLUP = [  # seed, N, d, w, nu, rho, nugget, n0, family, axis
    (610, 1200, 2, 1, 0.75, 0.3, 1e-4, 32, "matern", None),
    (611, 1000, 3, 1, 1.25, 0.3, 1e-4, 32, "matern", None),
    (612, 900, 2, 2, 0.75, 0.5, 1e-5, 32, "matern", [1.0, 4.0]),
    (613, 1100, 3, 1, None, 0.35, 1e-4, 32, "gaussian", None),
    (614, 1000, 3, 1, 2.5, 0.4, 1e-4, 32, "matern", [0.5, 2.0, 8.0]),
]


@pytest.mark.parametrize("seed,N,d,w,nu,rho,nug,n0,family,axis", BLUP)
def test_blup_tau_inf_matches_dense_oracle(pkg, seed, N, d, w, nu, rho, nug, n0, family, axis):
    P = wl.small_problem(seed, N, d, w, nu=1.5, rho=rho, nugget=nug, leaf_size=n0, M=200)
    kf = {"family": family, "axis": axis}
    ref = dense.dense_blup(P.points, P.Z, P.targets, w, nu, rho, nug, **kf)
    out = {}
    for prec, rtol in (("fp64", 1e-13), ("mixed", 1e-10)):
        ctx = pkg.Context(prec, leaf_size=n0, pcg_rtol=rtol, pcg_maxit=50000)
        ctx.build_basis(P.points, w)
        ctx.assemble(nu if nu else 1.5, rho, nug, math.inf, family=family, axis=axis)
        beta, info = ctx.solve(P.Z)
        assert info["converged"]
        out[prec] = ctx.predict(P.targets)
        ctx.close()
    assert rel(out["fp64"], ref["yhat"]) < 1e-9
    assert rel(out["mixed"], ref["yhat"]) < 1e-5


def test_matrix_free_general_nu_and_anisotropy(pkg):
    P = wl.small_problem(620, 1100, 3, 1, leaf_size=32, M=150)
    kf = {"family": "matern", "axis": [2.0, 0.5, 1.0]}
    ref = dense.dense_blup(P.points, P.Z, P.targets, 1, 0.75, 0.3, 1e-4, **kf)
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-5)):
        ctx = pkg.Context(prec, leaf_size=32, pcg_rtol=1e-12, pcg_maxit=50000, precond=False, matrix_free=True)
        ctx.build_basis(P.points, 1)
        ctx.assemble(0.75, 0.3, 1e-4, math.inf, **kf)
        ctx.solve(P.Z)
        assert rel(ctx.predict(P.targets), ref["yhat"]) < tol, prec
        ctx.close()


def test_finite_tau_general_nu_matches_multilevel_oracle(pkg):
    P = wl.small_problem(630, 1000, 3, 1, leaf_size=32, clustered=True, M=100)
    ctx = pkg.Context("fp64", leaf_size=32, pcg_rtol=1e-13, pcg_maxit=50000)
    ctx.build_basis(P.points, 1)
    ctx.assemble(1.25, 0.2, 1e-5, 2.0)
    beta, info = ctx.solve(P.Z)
    yhat = ctx.predict(P.targets)
    B = mlblup.setup(P.points, 1, 32)
    g, b, oi = mlblup.solve(B, P.points, P.Z, 1.25, 0.2, 1e-5, 2.0, exact=True)
    yref = mlblup.predict(B, P.points, g, b, P.targets, 1.25, 0.2)
    assert info["nnz"] == oi["nnz"]
    assert rel(yhat, yref) < 1e-9


@pytest.mark.parametrize("nu,family,axis", [(0.75, "matern", None), (1.25, "matern", [1.0, 2.0, 0.5]),
                                            (None, "gaussian", None)])
def test_grad_matches_dense_oracle(pkg, nu, family, axis):
    P = wl.small_problem(640, 900, 3, 1, leaf_size=32, M=150, with_y=True)
    ctx = pkg.Context("fp64", leaf_size=32, pcg_rtol=1e-12, pcg_maxit=50000)
    ctx.build_basis(P.points, 1)
    ctx.assemble(nu if nu else 1.5, 0.3, 1e-4, math.inf, family=family, axis=axis)
    ctx.solve(P.Z)
    got = ctx.grad(P.targets, P.y_targets)
    ref = og.grad_dense(P.points, P.Z, P.targets, P.y_targets, 1, nu, 0.3, 1e-4, family=family, axis=axis)
    ctx.close()
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-12)
