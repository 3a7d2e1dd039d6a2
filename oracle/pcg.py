"""Diagonally preconditioned conjugate gradients (Sec. 5.2 remark on P_W and
Sec. 6.2 "Predictor computation").

Solves A x = b with the preconditioner P = diag(A) (or I): P^{-1} A x = P^{-1} b.
The stopping test is on the residual of the *unpreconditioned* system,
||b - A x||_2 <= rtol ||b||_2 (the remark closing Sec. 6.2), using the
recursively updated residual r_k = b - A x_k.  Breakdown (p^T A p <= 0, which a
truncated C~_W can in principle produce) is reported, not hidden.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    rel_residual: float
    converged: bool
    breakdown: bool


def pcg(matvec, b: np.ndarray, diag: np.ndarray | None, rtol: float, maxit: int) -> PCGResult:
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return PCGResult(x, 0, 0.0, True, False)
    inv = (1.0 / diag) if diag is not None else np.ones_like(b)
    z = inv * r
    p = z.copy()
    rz = r @ z
    it = 0
    rel = 1.0
    while it < maxit:
        q = matvec(p)
        pq = p @ q
        if not pq > 0.0:
            return PCGResult(x, it, rel, False, True)
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = np.linalg.norm(r) / nb
        if rel <= rtol:
            return PCGResult(x, it, rel, True, False)
        z = inv * r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return PCGResult(x, it, rel, False, False)
