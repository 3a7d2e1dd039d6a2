"""Multilevel BLUP predictor (Sec. 5.2, eqs. Spatial:eqn1-3 and Spatial; Sec. 6.2).

    Z_W        = W Z
    C~_W g_W   = Z_W                 (PCG with P_W = diag(C~_W), or an exact solve)
    gamma-hat  = W^T g_W
    beta-hat   = (X^T X)^{-1} X^T (Z - C gamma-hat)      with the full, untruncated C
    Z-hat(x0)  = k(x0)^T beta-hat + c(x0)^T gamma-hat

``matvec="assembled"`` multiplies by the sparse C~_W of Algorithm 7;
``matvec="three_step"`` uses the three-step product of Sec. 6.2,
g -> W^T g -> C (W^T g) -> W C W^T g (the untruncated C_W).
"""
from __future__ import annotations

import math

import numpy as np
from .assemble import assemble, to_sparse
from .basis import build_basis
from .design import design_matrix
from .matern import kernel_matvec
from .pcg import pcg
from .tree import build_tree


def cov_matvec(points, v, nu, rho, nugget, **kf):
    """C v with C = [phi(r(x_i, x_j))] + eta I (kf: covariance family, axis weights)."""
    return kernel_matvec(points, points, v, nu, rho, **kf) + nugget * v


def setup(points, w, leaf_size, rank_rtol=None):
    tree = build_tree(points, leaf_size)
    return build_basis(points, tree, w, rank_rtol)


def solve(basis, points, Z, nu, rho, nugget, tau_factor, rtol=1e-10, maxit=10000,
          precond=True, matvec="assembled", exact=False, asm=None, **kf):
    ZW = basis.apply_W(Z)
    info = {}
    if matvec == "assembled":
        if asm is None:
            asm = assemble(basis, points, nu, rho, nugget, tau_factor, **kf)
        A = to_sparse(basis, asm)
        info["nnz"] = A.nnz
        info["asm"] = asm
        mv = lambda v: A @ v
        diag = A.diagonal()
    else:
        mv = lambda v: basis.apply_W(cov_matvec(points, basis.apply_Wt(v), nu, rho, nugget, **kf))
        diag = None
        A = None
    if exact:
        Ad = A.toarray() if A is not None else np.stack([mv(e) for e in np.eye(basis.nwav)], 1)
        gW = np.linalg.solve(Ad, ZW)
        info.update(iterations=0, rel_residual=float(np.linalg.norm(Ad @ gW - ZW) / np.linalg.norm(ZW)),
                    converged=True)
    else:
        res = pcg(mv, ZW, diag if precond else None, rtol, maxit)
        gW = res.x
        info.update(iterations=res.iterations, rel_residual=res.rel_residual,
                    converged=res.converged, breakdown=res.breakdown)
    gamma = basis.apply_Wt(gW)
    X = basis.X
    r = Z - cov_matvec(points, gamma, nu, rho, nugget, **kf)
    beta = np.linalg.solve(X.T @ X, X.T @ r)
    info["ZW"] = ZW
    info["gW"] = gW
    return gamma, beta, info


def predict(basis, points, gamma, beta, targets, nu, rho, **kf):
    """Eq. Spatial: k(x0)^T beta-hat + c(x0)^T gamma-hat (no nugget in c)."""
    K0 = design_matrix(targets, basis.w, basis.lo, basis.hi)
    return K0 @ beta + kernel_matvec(targets, points, gamma, nu, rho, **kf)


def blup(points, Z, targets, w, nu, rho, nugget, leaf_size, tau_factor=math.inf,
         rtol=1e-10, maxit=10000, precond=True, matvec="assembled", exact=False, **kf):
    basis = setup(points, w, leaf_size)
    gamma, beta, info = solve(basis, points, Z, nu, rho, nugget, tau_factor, rtol, maxit,
                              precond, matvec, exact, **kf)
    yhat = predict(basis, points, gamma, beta, targets, nu, rho, **kf)
    return {"basis": basis, "gamma": gamma, "beta": beta, "yhat": yhat, "info": info}
