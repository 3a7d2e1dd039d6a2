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

Any other smoothness nu > 0 is the definition itself, with the library's
modified Bessel function K_nu (scipy.special.kv) as one step.  The same
module gives the Gaussian kernel of the accuracy study (Sec. 8.2),
phi(r) = exp(-r^2 / (2 theta^2)) with theta passed as ``rho``, and the
anisotropic distance of Sec. 3, r(theta)^2 = (x - y)^T diag(theta) (x - y),
with the axis weights theta_k passed as ``axis`` (None: Euclidean).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import gammaln as _gammaln, kv as _kv

SUPPORTED_NU = (0.5, 1.5, 2.5)


def _s(r, nu, rho):
    return math.sqrt(2.0 * nu) * np.asarray(r, dtype=np.float64) / rho


def matern_kv(s, nu: float) -> np.ndarray:
    """The definition with the library's K_nu: phi = (s^nu K_nu(s)) / (Gamma(nu)
    2^(nu-1)) at s = sqrt(2 nu) r / rho, and phi(0) = 1 (the limit of s^nu
    K_nu(s) as s -> 0 is Gamma(nu) 2^(nu-1))."""
    s = np.asarray(s, dtype=np.float64)
    out = np.ones_like(s)
    pos = s > 0
    sp = s[pos]
    # in logarithms, so that Gamma(nu) 2^(nu-1) and s^nu K_nu(s) stay in range;
    # where K_nu(s) itself overflows, s is so small that phi = 1 to working
    # precision (1 - phi ~ s^(2 min(nu, 1)))
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        k = _kv(nu, sp)
        out[pos] = np.where(np.isfinite(k), np.exp(nu * np.log(sp) + np.log(k) - _gammaln(nu)
                                                   - (nu - 1.0) * math.log(2.0)), 1.0)
    return out


def dmatern_kv(s, nu: float) -> np.ndarray:
    """-s phi'(s) from the definition: d/ds [s^nu K_nu(s)] = -s^nu K_{nu-1}(s)
    (A&S 9.6.28), so -s phi'(s) = s^(nu+1) K_{nu-1}(s) / (Gamma(nu) 2^(nu-1))."""
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros_like(s)
    pos = s > 0
    sp = s[pos]
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        k = _kv(nu - 1.0, sp)
        # where K_{nu-1}(s) overflows, -s phi'(s) ~ s^2 (nu > 1) or s^(2 nu) is below working precision
        out[pos] = np.where(np.isfinite(k), np.exp((nu + 1.0) * np.log(sp) + np.log(k) - _gammaln(nu)
                                                   - (nu - 1.0) * math.log(2.0)), 0.0)
    return out


def matern(r, nu: float, rho: float, family: str = "matern") -> np.ndarray:
    """phi(r; nu, rho) (unit variance): closed forms at nu = 1/2, 3/2, 5/2, the
    definition with K_nu otherwise; family="gaussian": exp(-r^2 / (2 rho^2))."""
    if family == "gaussian":
        t = np.asarray(r, dtype=np.float64) / rho
        return np.exp(-0.5 * t * t)
    if family != "matern":
        raise ValueError(f"unknown covariance family {family!r}")
    s = _s(r, nu, rho)
    e = np.exp(-s)
    if nu == 0.5:
        return e
    if nu == 1.5:
        return (1.0 + s) * e
    if nu == 2.5:
        return (1.0 + s + s * s / 3.0) * e
    if not nu > 0:
        raise ValueError(f"nu={nu} must be positive")
    return matern_kv(s, nu)


def dmatern_dlogrho(r, nu: float, rho: float, family: str = "matern") -> np.ndarray:
    """d phi / d log(rho).  Since s is proportional to 1/rho, ds/dlog(rho) = -s,
    so the derivative is -s phi'(s):

        nu = 1/2 : s e^{-s}
        nu = 3/2 : s^2 e^{-s}
        nu = 5/2 : (s^2/3)(1 + s) e^{-s}
        other nu : s^(nu+1) K_{nu-1}(s) / (Gamma(nu) 2^(nu-1))
        Gaussian : (r/rho)^2 exp(-r^2 / (2 rho^2))
    """
    if family == "gaussian":
        t = np.asarray(r, dtype=np.float64) / rho
        return t * t * np.exp(-0.5 * t * t)
    s = _s(r, nu, rho)
    e = np.exp(-s)
    if nu == 0.5:
        return s * e
    if nu == 1.5:
        return s * s * e
    if nu == 2.5:
        return (s * s / 3.0) * (1.0 + s) * e
    return dmatern_kv(s, nu)


def distances(x: np.ndarray, y: np.ndarray, axis=None) -> np.ndarray:
    """Distances between rows of x (m,d) and y (n,d), formed from the coordinate
    differences (not from |x|^2 + |y|^2 - 2 x.y).  With axis weights theta_k
    (Sec. 3): r^2 = sum_k theta_k (x_k - y_k)^2; None: Euclidean."""
    acc = np.zeros((x.shape[0], y.shape[0]))
    for k in range(x.shape[1]):
        diff = x[:, k][:, None] - y[:, k][None, :]
        acc += diff * diff if axis is None else axis[k] * (diff * diff)
    return np.sqrt(acc)


def kernel_matrix(x: np.ndarray, y: np.ndarray, nu: float, rho: float, family: str = "matern",
                  axis=None) -> np.ndarray:
    """[phi(r(x_i, y_j))]_{ij} (no nugget)."""
    return matern(distances(x, y, axis), nu, rho, family)


def kernel_matvec(x: np.ndarray, y: np.ndarray, v: np.ndarray, nu: float, rho: float,
                  chunk: int = 2048, family: str = "matern", axis=None) -> np.ndarray:
    """sum_j phi(r(x_i, y_j)) v_j, in row chunks (no nugget)."""
    out = np.empty(x.shape[0])
    for s in range(0, x.shape[0], chunk):
        out[s:s + chunk] = kernel_matrix(x[s:s + chunk], y, nu, rho, family, axis) @ v
    return out


def covariance(x: np.ndarray, nu: float, rho: float, nugget: float, family: str = "matern",
               axis=None) -> np.ndarray:
    """Covariance matrix C of the observations at x: phi(r(x_i, x_j)) + eta delta_ij."""
    c = kernel_matrix(x, x, nu, rho, family, axis)
    c[np.diag_indices_from(c)] += nugget
    return c
