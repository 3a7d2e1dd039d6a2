"""Gradient of a held-out prediction loss in log(rho) and log(nugget).

The paper estimates theta by maximum likelihood and has no gradient of the
predictor; this is the plain adjoint of its BLUP equations.  With
K = [[C, X], [X^T, 0]] and K [gamma; beta] = [Z; 0] (eq. Spatial:problem),
predictions Y-hat_k = c(x0_k)^T gamma + k(x0_k)^T beta (eq. Spatial) and the
loss L = (1/M) sum_k (Y-hat_k - y_k)^2:

    g_k      = 2 (Y-hat_k - y_k) / M
    a        = sum_k g_k c(x0_k),   b = sum_k g_k k(x0_k)
    K [lambda; mu] = [a; b]                          (adjoint system; K is symmetric)
    dL/dtheta = sum_k g_k (dc_k/dtheta)^T gamma - lambda^T (dC/dtheta) gamma

with dC/dlog(rho) = [d phi/d log rho (|x_i - x_j|)], dC/dlog(eta) = eta I, and
targets free of nugget (dc/dlog(eta) = 0).

The multilevel adjoint solves the same system the way eqs. Spatial:eqn1-2
solve the forward one: lambda_0 = X (X^T X)^{-1} b satisfies X^T lambda_0 = b
and W lambda_0 = 0, and lambda = lambda_0 + W^T lambda_W with
C_W lambda_W = W (a - C lambda_0).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import cho_factor, cho_solve

from . import mlblup
from .design import box, design_matrix
from .matern import covariance, dmatern_dlogrho, distances, kernel_matrix
from .pcg import pcg


def loss_dense(points, Z, targets, y, w, nu, rho, nugget, **kf):
    from .dense import dense_blup
    r = dense_blup(points, Z, targets, w, nu, rho, nugget, **kf)
    return float(np.mean((r["yhat"] - y) ** 2))


def grad_dense(points, Z, targets, y, w, nu, rho, nugget, family="matern", axis=None):
    kf = {"family": family, "axis": axis}
    lo, hi = box(points)
    X = design_matrix(points, w, lo, hi)
    C = covariance(points, nu, rho, nugget, **kf)
    cf = cho_factor(C, lower=True)
    CiX = cho_solve(cf, X)
    beta = np.linalg.solve(X.T @ CiX, X.T @ cho_solve(cf, Z))
    gamma = cho_solve(cf, Z - X @ beta)
    c0 = kernel_matrix(targets, points, nu, rho, **kf)
    K0 = design_matrix(targets, w, lo, hi)
    yhat = c0 @ gamma + K0 @ beta
    M = targets.shape[0]
    loss = float(np.mean((yhat - y) ** 2))
    g = 2.0 * (yhat - y) / M
    a, b = c0.T @ g, K0.T @ g
    mu = np.linalg.solve(X.T @ CiX, X.T @ cho_solve(cf, a) - b)
    lam = cho_solve(cf, a - X @ mu)
    dC = dmatern_dlogrho(distances(points, points, axis), nu, rho, family)
    dc0 = dmatern_dlogrho(distances(targets, points, axis), nu, rho, family)
    d_logrho = g @ (dc0 @ gamma) - lam @ (dC @ gamma)
    d_lognug = -nugget * (lam @ gamma)
    return loss, float(d_logrho), float(d_lognug)


def grad_multilevel(points, Z, targets, y, w, nu, rho, nugget, leaf_size, tau_factor=math.inf,
                    rtol=1e-12, maxit=10000):
    basis = mlblup.setup(points, w, leaf_size)
    gamma, beta, info = mlblup.solve(basis, points, Z, nu, rho, nugget, tau_factor, rtol, maxit)
    from .assemble import to_sparse
    A = to_sparse(basis, info["asm"])
    K0 = design_matrix(targets, w, basis.lo, basis.hi)
    c0 = kernel_matrix(targets, points, nu, rho)
    yhat = K0 @ beta + c0 @ gamma
    M = targets.shape[0]
    loss = float(np.mean((yhat - y) ** 2))
    g = 2.0 * (yhat - y) / M
    a, b = c0.T @ g, K0.T @ g
    X = basis.X
    lam0 = X @ np.linalg.solve(X.T @ X, b)
    rhs = basis.apply_W(a - mlblup.cov_matvec(points, lam0, nu, rho, nugget))
    res = pcg(lambda v: A @ v, rhs, A.diagonal(), rtol, maxit)
    lam = lam0 + basis.apply_Wt(res.x)
    dC = dmatern_dlogrho(distances(points, points), nu, rho)
    dc0 = dmatern_dlogrho(distances(targets, points), nu, rho)
    d_logrho = g @ (dc0 @ gamma) - lam @ (dC @ gamma)
    d_lognug = -nugget * (lam @ gamma)
    return loss, float(d_logrho), float(d_lognug)
