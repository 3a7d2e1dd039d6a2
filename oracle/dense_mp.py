"""Dense BLUP in extended precision for the ill-conditioned accuracy study
(Sec. 8.2, Table 5), where the covariance matrix of the Gaussian kernel has a
condition number near 1e19 and the FP64 formulae lose every digit.

The paper's reference solution is computed with 52 significant digits; this
is the same definition -- the saddle-point system of eq. Spatial:problem,

    [[C, X], [X^T, 0]] [gamma; beta] = [Z; 0],   Z-hat(x0) = k(x0)^T beta + c(x0)^T gamma,

solved by Gaussian elimination with partial pivoting (mpmath's LU, one
library step) at ``dps`` decimal digits (50 by default).  The design matrix is
the oracle's (total-degree monomials of the box-scaled coordinates, graded
order), formed in the same precision from the FP64 inputs, which convert to
mpmath numbers exactly.  TEST INFRASTRUCTURE ONLY, like the rest of the oracle.
"""
from __future__ import annotations

import numpy as np

from .design import box, exponents


def _mp():
    import mpmath
    return mpmath


def _design(mp, x, lo, hi, w):
    d = x.shape[1]
    ex = exponents(d, w)
    rows = []
    for i in range(x.shape[0]):
        u = [mp.mpf(2) * (mp.mpf(float(x[i, c])) - mp.mpf(float(lo[c]))) / (mp.mpf(float(hi[c])) - mp.mpf(float(lo[c])))
             - 1 for c in range(d)]
        row = []
        for a in ex:
            v = mp.mpf(1)
            for c in range(d):
                v *= u[c] ** a[c]
            row.append(v)
        rows.append(row)
    return rows


def gaussian_kernel(mp, x, y, theta):
    """[exp(-|x_i - y_j|^2 / (2 theta^2))] in mpmath numbers."""
    t2 = 2 * mp.mpf(float(theta)) ** 2
    out = []
    for i in range(x.shape[0]):
        xi = [mp.mpf(float(v)) for v in x[i]]
        row = []
        for j in range(y.shape[0]):
            r2 = sum((xi[c] - mp.mpf(float(y[j, c]))) ** 2 for c in range(x.shape[1]))
            row.append(mp.exp(-r2 / t2))
        out.append(row)
    return out


def dense_blup_mp(points, Z, targets, w, theta, nugget=0.0, dps=50):
    """Gaussian-kernel BLUP at ``dps`` digits.  Returns float64 arrays
    (yhat, beta, gamma) and the saddle-point residual norm (in mpmath)."""
    mp = _mp()
    with mp.workdps(dps):
        lo, hi = box(points)
        X = _design(mp, points, lo, hi, w)
        C = gaussian_kernel(mp, points, points, theta)
        N, p = len(X), len(X[0])
        K = mp.zeros(N + p, N + p)
        for i in range(N):
            for j in range(N):
                K[i, j] = C[i][j] + (mp.mpf(float(nugget)) if i == j else 0)
            for j in range(p):
                K[i, N + j] = X[i][j]
                K[N + j, i] = X[i][j]
        rhs = mp.matrix([mp.mpf(float(v)) for v in Z] + [0] * p)
        sol = mp.lu_solve(K, rhs)
        res = mp.norm(K * sol - rhs)
        gamma = [sol[i] for i in range(N)]
        beta = [sol[N + j] for j in range(p)]
        K0 = _design(mp, targets, lo, hi, w)
        c0 = gaussian_kernel(mp, targets, points, theta)
        yhat = [sum(K0[k][j] * beta[j] for j in range(p)) + sum(c0[k][i] * gamma[i] for i in range(N))
                for k in range(len(K0))]
        return (np.array([float(v) for v in yhat]), np.array([float(v) for v in beta]),
                np.array([float(v) for v in gamma]), res)
