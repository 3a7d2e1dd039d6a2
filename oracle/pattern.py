"""Distance criterion and tree search for the sparse C~_W (Sec. 4.1, Algorithms 4-6).

The text defines the criterion: extend the source cell's point bounding box by
tau_{i,j} on every axis, [x_k^min - tau, x_k^max + tau], and include every
target cell at the requested depth that meets it.  Algorithms 4-6 find those
cells by descending from the root: at a node with split (v, thr) go left
unless every source point has x.v - tau > thr, go right unless every source
point has x.v + tau <= thr (the text's form; Algorithm 6 prints the right rule
with +tau, which contradicts the text, and the text is used).

Readings:

* A target cell "meets" the grown box when its own points' bounding box does
  (the search reaches every such cell, since a cell's points lie inside its kd
  region; its result is filtered by this box test).  The test is symmetric in
  the two cells, so the pattern of C~_W is symmetric.
* tau_{i,j}: the paper sets one distance per level pair, tau_{i,j} =
  2^{(t-i)/2} 2^{(t-j)/2} tau (Sec. 8.1); the configurations state "tau = c cell
  diameters".  Here tau_{i,j} = c * sqrt(Dbar_i * Dbar_j) with Dbar_l the mean,
  over the cells of level l, of the Euclidean diagonal of the cell's point
  bounding box (summed cell by cell in order, then divided by the count) --
  the geometric mean of the two levels' cell sizes in place of the paper's
  sqrt(2^{t-i} 2^{t-j}).  c = inf keeps every pair (dense C_W).
* Target depth j >= i (Remark after Algorithm 6: only blocks j >= i are
  computed, the rest by symmetry); all leaves sit at depth t, so the search
  always reaches depth j.

Floating point: D is accumulated axis by axis in order, Dbar cell by cell in
order, tau = c * sqrt(Dbar_i Dbar_j), and a pair is excluded iff on some axis
lo_q - hi_m > tau or lo_m - hi_q > tau.
"""
from __future__ import annotations

import math

import numpy as np

from .tree import Tree


def diameters(tree: Tree, l: int) -> np.ndarray:
    lo, hi = tree.lo[l], tree.hi[l]
    acc = np.zeros(lo.shape[0])
    for k in range(lo.shape[1]):
        span = hi[:, k] - lo[:, k]
        acc = acc + span * span
    return np.sqrt(acc)


def level_mean_diameter(tree: Tree, l: int) -> float:
    acc = 0.0
    for v in diameters(tree, l).tolist():
        acc = acc + v
    return acc / tree.ncells(l)


def tau_levels(tree: Tree, i: int, j: int, c: float) -> float:
    if math.isinf(c):
        return math.inf
    return c * math.sqrt(level_mean_diameter(tree, i) * level_mean_diameter(tree, j))


def box_admissible(lo_m, hi_m, lo_q, hi_q, tau) -> np.ndarray:
    """True where the tau-grown box of m meets the box of q (broadcasting)."""
    ok = np.ones(np.broadcast(lo_m[..., 0], lo_q[..., 0]).shape, dtype=bool)
    for k in range(lo_m.shape[-1]):
        ok &= ~((lo_q[..., k] - hi_m[..., k]) > tau)
        ok &= ~((lo_m[..., k] - hi_q[..., k]) > tau)
    return ok


def level_pair_bruteforce(tree: Tree, i: int, j: int, c: float) -> np.ndarray:
    """Boolean (2^i, 2^j) matrix of admissible (m, q) pairs by testing all pairs."""
    tau = tau_levels(tree, i, j, c)
    return box_admissible(tree.lo[i][:, None, :], tree.hi[i][:, None, :],
                          tree.lo[j][None, :, :], tree.hi[j][None, :, :], tau)


def search_tree(tree: Tree, lo_K: np.ndarray, hi_K: np.ndarray, target_depth: int,
                tau: float) -> list[int]:
    """Algorithms 4-6 (SearchTree, LocalSearchTree, ChooseLeft/RightRule): cells at the
    target depth whose kd region meets the tau-grown extent of the source points
    (given by their per-axis min lo_K and max hi_K)."""
    found: list[int] = []

    def local(l: int, k: int):
        if l == target_depth:
            found.append(k)
            return
        if l == tree.t:                      # a leaf above the target depth
            return
        ax, th = tree.axis[l][k], tree.thr[l][k]
        if not (lo_K[ax] - tau > th):        # not every x.v - tau > thr: left side reachable
            local(l + 1, 2 * k)
        if not (hi_K[ax] + tau <= th):       # not every x.v + tau <= thr: right side reachable
            local(l + 1, 2 * k + 1)

    local(0, 0)
    return found


def level_pair_search(tree: Tree, i: int, j: int, c: float) -> np.ndarray:
    """Pattern of level pair (i, j) by Algorithms 4-6 followed by the box test."""
    tau = tau_levels(tree, i, j, c)
    out = np.zeros((tree.ncells(i), tree.ncells(j)), dtype=bool)
    for m in range(tree.ncells(i)):
        for q in search_tree(tree, tree.lo[i][m], tree.hi[i][m], j, tau):
            out[m, q] = bool(box_admissible(tree.lo[i][m], tree.hi[i][m],
                                            tree.lo[j][q], tree.hi[j][q], tau))
    return out


def pattern(tree: Tree, c: float, method: str = "search") -> dict[tuple[int, int], np.ndarray]:
    """{(i, j): bool (2^i, 2^j)} for all level pairs i <= j."""
    f = level_pair_search if method == "search" else level_pair_bruteforce
    return {(i, j): f(tree, i, j, c) for i in range(tree.t + 1) for j in range(i, tree.t + 1)}
