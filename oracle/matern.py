"""Matern covariance, Def. "Matern covariance function" (Sec. 3.1).

phi(r) = (sqrt(2 nu) r / rho)^nu K_nu(sqrt(2 nu) r / rho) / (Gamma(nu) 2^(nu-1)).

The half-integer remark that follows the definition is garbled in the source
(its sum starts at k = 1 and carries a factor (n+1)!), so the closed forms here
are derived from the definition itself with the textbook half-integer Bessel
functions K_{n+1/2}(s) = sqrt(pi/(2s)) e^{-s} sum_k (n+k)!/(k!(n-k)!) (2s)^{-k}:
with s = sqrt(2 nu) r / rho,

    nu = 1/2 : e^{-s}
    nu = 3/2 : (1 + s) e^{-s}
    nu = 5/2 : (1 + s + s^2/3) e^{-s}

Unit variance: phi(0) = 1.  The covariance matrix of the observations adds
the nugget eta on its diagonal (C <- C + eta I on data points only).
"""
from __future__ import annotations

import math

import numpy as np

SUPPORTED_NU = (0.5, 1.5, 2.5)


def _s(r, nu, rho):
    return math.sqrt(2.0 * nu) * np.asarray(r, dtype=np.float64) / rho


def matern(r, nu: float, rho: float) -> np.ndarray:
    """phi(r; nu, rho) for nu in {1/2, 3/2, 5/2} (unit variance)."""
    s = _s(r, nu, rho)
    e = np.exp(-s)
    if nu == 0.5:
        return e
    if nu == 1.5:
        return (1.0 + s) * e
    if nu == 2.5:
        return (1.0 + s + s * s / 3.0) * e
    raise ValueError(f"nu={nu} not supported (half-integer 1/2, 3/2, 5/2 only)")


def dmatern_dlogrho(r, nu: float, rho: float) -> np.ndarray:
    """d phi / d log(rho).  Since s is proportional to 1/rho, ds/dlog(rho) = -s,
    so the derivative is -s phi'(s):

        nu = 1/2 : s e^{-s}
        nu = 3/2 : s^2 e^{-s}
        nu = 5/2 : (s^2/3)(1 + s) e^{-s}
    """
    s = _s(r, nu, rho)
    e = np.exp(-s)
    if nu == 0.5:
        return s * e
    if nu == 1.5:
        return s * s * e
    if nu == 2.5:
        return (s * s / 3.0) * (1.0 + s) * e
    raise ValueError(f"nu={nu} not supported")


def distances(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Euclidean distances between rows of x (m,d) and y (n,d), formed from the
    coordinate differences (not from |x|^2 + |y|^2 - 2 x.y)."""
    acc = np.zeros((x.shape[0], y.shape[0]))
    for k in range(x.shape[1]):
        diff = x[:, k][:, None] - y[:, k][None, :]
        acc += diff * diff
    return np.sqrt(acc)


def kernel_matrix(x: np.ndarray, y: np.ndarray, nu: float, rho: float) -> np.ndarray:
    """[phi(|x_i - y_j|)]_{ij} (no nugget)."""
    return matern(distances(x, y), nu, rho)


def kernel_matvec(x: np.ndarray, y: np.ndarray, v: np.ndarray, nu: float, rho: float,
                  chunk: int = 2048) -> np.ndarray:
    """sum_j phi(|x_i - y_j|) v_j, in row chunks (no nugget)."""
    out = np.empty(x.shape[0])
    for s in range(0, x.shape[0], chunk):
        out[s:s + chunk] = kernel_matrix(x[s:s + chunk], y, nu, rho) @ v
    return out


def covariance(x: np.ndarray, nu: float, rho: float, nugget: float) -> np.ndarray:
    """Covariance matrix C of the observations at x: phi(|x_i - x_j|) + eta delta_ij."""
    c = kernel_matrix(x, x, nu, rho)
    c[np.diag_indices_from(c)] += nugget
    return c
