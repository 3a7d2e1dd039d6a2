"""kd-tree of the observation locations (Sec. 3.1, Algorithms 1-3).

Rule (Algorithm 1): in a cell, take the coordinate axis of maximal variance of
the cell's points, project on it and split at the median of the projections.
InitialTree / MakeTree (Algorithms 2, 3): start from the root cell holding all
of S and split recursively, left before right.

Readings (the algorithm text is inconsistent on these points):

* Leaf size.  MakeTree stops at |S_T| < n0 while the text and Fig. 1 speak of
  leaves holding *at most* n0 points.  Here a cell splits while it holds more
  than n0 points.  The median split keeps the sizes of all cells of one level
  within one point of each other (floor/ceil of N / 2^l), so every cell is
  split down to the common depth t = min{ t : ceil(N / 2^t) <= n0 }; all leaves
  sit at depth t, as in Fig. 1.
* Variance: population variance (divide by the cell size); ties between axes
  go to the lowest axis index.
* Median: the cell's points are ordered by (coordinate on the split axis,
  original index); the first floor(s/2) go left, the rest right; the stored
  threshold is the coordinate of the last left point, so Rule(x) = x.v <= thr
  holds for every left point.
* Node numbering: level order (cell k of level l has children 2k and 2k+1 of
  level l+1) instead of the depth-first numbering of MakeTree; the tree shape
  is the same.  Points are stored permuted so that every cell is a contiguous
  range [begin, end) of the permutation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Tree:
    t: int                         # depth of the leaves (root is level 0)
    perm: np.ndarray               # (N,) original index of the point at each position
    begin: list[np.ndarray]        # begin[l][k]: first position of cell k of level l
    end: list[np.ndarray]          # end[l][k]: one past the last position
    axis: list[np.ndarray]         # split axis of cell k of level l (levels < t)
    thr: list[np.ndarray]          # split threshold (levels < t)
    lo: list[np.ndarray]           # (2^l, d) bounding box of the cell's points
    hi: list[np.ndarray]

    @property
    def levels(self) -> int:
        return self.t + 1

    def ncells(self, l: int) -> int:
        return len(self.begin[l])


def depth_for(N: int, n0: int) -> int:
    t = 0
    while -(-N // (1 << t)) > n0:
        t += 1
    return t


def rule(pts: np.ndarray, orig: np.ndarray):
    """Algorithm 1 on one cell: returns (axis, order, threshold) where ``order``
    sorts the cell by (projection, original index) and the first half goes left."""
    var = pts.var(axis=0)
    axis = int(np.argmax(var))
    order = np.lexsort((orig, pts[:, axis]))
    h = pts.shape[0] // 2
    thr = pts[order[h - 1], axis] if h > 0 else -np.inf
    return axis, order, thr


def build_tree(points: np.ndarray, n0: int) -> Tree:
    """Algorithms 2-3 (level by level; see the module docstring)."""
    N, d = points.shape
    t = depth_for(N, n0)
    perm = np.arange(N)
    begin = [np.array([0])]
    end = [np.array([N])]
    axis: list[np.ndarray] = []
    thr: list[np.ndarray] = []
    for l in range(t):
        nb, ne = [], []
        ax_l = np.zeros(len(begin[l]), dtype=np.int64)
        th_l = np.zeros(len(begin[l]))
        for k, (b, e) in enumerate(zip(begin[l], end[l])):
            idx = perm[b:e]
            a, order, th = rule(points[idx], idx)
            perm[b:e] = idx[order]
            h = (e - b) // 2
            ax_l[k], th_l[k] = a, th
            nb += [b, b + h]
            ne += [b + h, e]
        axis.append(ax_l)
        thr.append(th_l)
        begin.append(np.array(nb))
        end.append(np.array(ne))
    lo, hi = [], []
    for l in range(t + 1):
        lo.append(np.stack([points[perm[b:e]].min(axis=0) for b, e in zip(begin[l], end[l])]))
        hi.append(np.stack([points[perm[b:e]].max(axis=0) for b, e in zip(begin[l], end[l])]))
    return Tree(t, perm, begin, end, axis, thr, lo, hi)
