"""Classic single-level BLUP (Sec. 2, eqs. GLSbeta and KrigBLUP; Sec. 5.2,
eqs. Spatial:problem and Spatial).

    beta-hat  = (X^T C^{-1} X)^{-1} X^T C^{-1} Z
    gamma-hat = C^{-1} (Z - X beta-hat)
    Z-hat(x0) = k(x0)^T beta-hat + c(x0)^T gamma-hat

computed with a Cholesky factorisation of C (library routines as single
steps).  C is the covariance of the observations, nugget included; the
cross-covariance c(x0) between data and a target carries no nugget.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cho_factor, cho_solve

from .design import box, design_matrix
from .matern import covariance, kernel_matrix


def dense_blup(points, Z, targets, w, nu, rho, nugget, **kf):
    """kf: covariance family and axis weights (matern.kernel_matrix)."""
    lo, hi = box(points)
    X = design_matrix(points, w, lo, hi)
    C = covariance(points, nu, rho, nugget, **kf)
    cf = cho_factor(C, lower=True)
    CiX = cho_solve(cf, X)
    CiZ = cho_solve(cf, Z)
    beta = np.linalg.solve(X.T @ CiX, X.T @ CiZ)
    gamma = cho_solve(cf, Z - X @ beta)
    K0 = design_matrix(targets, w, lo, hi)
    c0 = kernel_matrix(targets, points, nu, rho, **kf)
    yhat = K0 @ beta + c0 @ gamma
    return {"beta": beta, "gamma": gamma, "yhat": yhat, "X": X, "C": C}


def saddle_point_solve(points, Z, w, nu, rho, nugget, **kf):
    """Direct solve of [[C, X], [X^T, 0]] [gamma; beta] = [Z; 0]."""
    lo, hi = box(points)
    X = design_matrix(points, w, lo, hi)
    C = covariance(points, nu, rho, nugget, **kf)
    N, p = X.shape
    K = np.zeros((N + p, N + p))
    K[:N, :N] = C
    K[:N, N:] = X
    K[N:, :N] = X.T
    sol = np.linalg.solve(K, np.concatenate([Z, np.zeros(p)]))
    return sol[:N], sol[N:]


def mse_at(points, targets, w, nu, rho, nugget, **kf):
    """Kriging mean squared error at targets (Sec. 5.2, after eq. Spatial)."""
    lo, hi = box(points)
    X = design_matrix(points, w, lo, hi)
    C = covariance(points, nu, rho, nugget, **kf)
    cf = cho_factor(C, lower=True)
    c0 = kernel_matrix(points, targets, nu, rho, **kf)
    Cic = cho_solve(cf, c0)
    A = X.T @ cho_solve(cf, X)
    K0 = design_matrix(targets, w, lo, hi)
    u = X.T @ Cic - K0.T
    return 1.0 + np.einsum("ik,ik->k", u, np.linalg.solve(A, u)) - np.einsum("ik,ik->k", c0, Cic)
