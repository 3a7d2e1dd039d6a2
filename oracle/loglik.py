"""Multilevel log-likelihood (Sec. 5.1, the reduced likelihood of the full
transform, n = 0) and a stochastic Lanczos quadrature estimate of its
log-determinant.  Test infrastructure: plain numpy FP64, slow, for checking.

    l_W(theta) = -(N~/2) log(2 pi) - (1/2) log det C_W - (1/2) Z_W^T C_W^{-1} Z_W,
    Z_W = W Z,  N~ = N - p.

The paper obtains log det C_W from a sparse Cholesky factorisation; the GPU
path estimates it by stochastic Lanczos quadrature (Ubaru, Chen and Saad,
SIAM J. Matrix Anal. Appl. 38, 2017): for probe vectors v_i,

    log det A = tr log A ~ (1/m) sum_i |v_i|^2 sum_j (e_1^T u_j)^2 log theta_j,

with (theta_j, u_j) the eigenpairs of the k x k Lanczos tridiagonal started at
v_i / |v_i|.  Here the Lanczos vectors are fully reorthogonalised (classical
Gram-Schmidt against all previous vectors, twice), as on the GPU.
"""
from __future__ import annotations

import math

import numpy as np

from .assemble import assemble, to_sparse


def lanczos_tridiagonal(A: np.ndarray, v: np.ndarray, k: int):
    """k steps of Lanczos on the symmetric matrix A from v / |v|, with full
    reorthogonalisation; returns (alpha, beta) of the tridiagonal (stopping
    early at an invariant subspace)."""
    n = v.shape[0]
    k = min(k, n)
    Q = np.zeros((k + 1, n))
    Q[0] = v / np.linalg.norm(v)
    alpha, beta = [], []
    for j in range(k):
        w = A @ Q[j]
        c = Q[: j + 1] @ w
        alpha.append(c[j])
        w = w - Q[: j + 1].T @ c
        w = w - Q[: j + 1].T @ (Q[: j + 1] @ w)
        b = np.linalg.norm(w)
        if j < k - 1 and not b > 1e-12 * abs(alpha[-1]):
            break
        beta.append(b)
        Q[j + 1] = w / b if b > 0 else 0.0
    m = len(alpha)
    return np.array(alpha), np.array(beta[: m - 1])


def slq_logdet(A: np.ndarray, probes: np.ndarray, k: int) -> float:
    """Stochastic Lanczos quadrature estimate of log det A over the probe rows."""
    total = 0.0
    for v in probes:
        a, b = lanczos_tridiagonal(A, v, k)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        theta, U = np.linalg.eigh(T)
        if np.any(theta <= 0):
            raise np.linalg.LinAlgError("not positive definite")
        total += float(v @ v) * float(np.sum(U[0] ** 2 * np.log(theta)))
    return total / max(len(probes), 1)


def cw_dense(basis, points, nu, rho, nugget, tau_factor=math.inf) -> np.ndarray:
    """C~_W of Algorithm 7 as a dense matrix (small problems only)."""
    return to_sparse(basis, assemble(basis, points, nu, rho, nugget, tau_factor)).toarray()


def multilevel_loglik(basis, points, Z, nu, rho, nugget, tau_factor=math.inf, probes=None, steps=30):
    """(l_W, log det, quadratic form); log det exact (slogdet) unless probes
    (data-space vectors, rows) are given, then the SLQ estimate with W z."""
    A = cw_dense(basis, points, nu, rho, nugget, tau_factor)
    ZW = basis.apply_W(Z)
    quad = float(ZW @ np.linalg.solve(A, ZW))
    if probes is None:
        sign, logdet = np.linalg.slogdet(A)
        if sign <= 0:
            raise np.linalg.LinAlgError("C~_W is not positive definite")
    else:
        V = np.stack([basis.apply_W(z) for z in probes])
        logdet = slq_logdet(A, V, steps)
    n = ZW.shape[0]
    return -0.5 * (n * math.log(2.0 * math.pi) + logdet + quad), float(logdet), quad
