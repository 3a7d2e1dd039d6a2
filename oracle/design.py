"""Total-degree design matrix (Sec. 2, the monomial set Q^d_w).

Q^d_w = { x^alpha : |alpha| <= w }, with p(d, w) = binomial(d + w, w) members.
X = (k(x_1) ... k(x_N))^T with k(x) the vector of these monomials.

Reading: the paper assumes the locations lie in [-1, 1]^d "without loss of
generality"; the data here lie in [0, 1]^d or wherever the user puts them, so
the coordinates are first mapped affinely onto [-1, 1]^d by the bounding box of
the observation locations, u = 2 (x - lo) / (hi - lo) - 1 (u = 0 on an axis
with hi == lo).  The span of the TD monomials is invariant under this map, so
W, gamma-hat and the predictions do not depend on it; beta-hat is reported in
this scaled monomial basis.  Monomial order: graded, and within one degree
lexicographically decreasing in the exponent vector (1, x1, ..., xd, x1^2,
x1 x2, ...).
"""
from __future__ import annotations

import math

import numpy as np


def exponents(d: int, w: int) -> list[tuple[int, ...]]:
    """Exponent vectors alpha with |alpha| <= w in graded lex-decreasing order."""
    out: list[tuple[int, ...]] = []

    def rec(prefix, remaining, k):
        if k == d - 1:
            out_deg.append(tuple(prefix + [remaining]))
            return
        for a in range(remaining, -1, -1):
            rec(prefix + [a], remaining - a, k + 1)

    for deg in range(w + 1):
        out_deg: list[tuple[int, ...]] = []
        if d == 0:
            continue
        rec([], deg, 0)
        out.extend(out_deg)
    return out


def num_monomials(d: int, w: int) -> int:
    return math.comb(d + w, w)


def box(points: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    return points.min(axis=0), points.max(axis=0)


def scale(x: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Affine map of the data bounding box [lo, hi] onto [-1, 1]^d."""
    span = hi - lo
    u = np.zeros_like(x, dtype=np.float64)
    ok = span > 0
    u[:, ok] = 2.0 * (x[:, ok] - lo[ok]) / span[ok] - 1.0
    return u


def design_matrix(x: np.ndarray, w: int, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """X[i, j] = u_i^{alpha_j} with u the box-scaled coordinates of x_i."""
    u = scale(x, lo, hi)
    alphas = exponents(x.shape[1], w)
    X = np.ones((x.shape[0], len(alphas)))
    for j, alpha in enumerate(alphas):
        for k, a in enumerate(alpha):
            for _ in range(a):
                X[:, j] *= u[:, k]
    return X
