"""Multilevel basis (Sec. 3.1, construction steps 1-5, and the operators W, L).

Bottom-up over the kd-tree.  For a leaf cell with s points the local basis
vectors are the unit vectors of its points; for an internal cell they are the
scaling vectors of its two children.  With B the matrix of these local basis
vectors (on the points), form the moment matrix M = X^T B (p x s), take its SVD
M = U D V^T, and split the columns of V: the first a (a = numerical rank of M)
give the scaling vectors phi = B V[:, :a], the remaining s - a give the
wavelets psi = B V[:, a:], which satisfy X^T psi = 0 (eq.
hbconstruction:eqn1).  At the root the a = p scaling vectors span the column
space of X; they are the rows of L.  W stacks the wavelets finest level first,
W = [W_t; ...; W_0], cells left to right within a level.

Reading: the numerical rank is a = #{sigma_i > rtol * sigma_max} with
rtol = 10 * max(p, s) * 2^-52 unless given; the root must reach a = p (X of
full column rank), else ``RankDeficient`` is raised.

Each cell keeps its scaling and wavelet vectors explicitly on its points
(n_c x a_c and n_c x k_c) -- the plain representation, O(N (n0 + t p)) numbers.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .design import box, design_matrix
from .tree import Tree


class RankDeficient(ValueError):
    pass


@dataclass
class Basis:
    tree: Tree
    p: int
    w: int                           # total degree of the trend space
    X: np.ndarray                    # (N, p) design matrix, user order
    lo: np.ndarray                   # data bounding box used to scale X
    hi: np.ndarray
    phi: list[list[np.ndarray]]      # phi[l][k]: (n_c, a_c) scaling vectors on the cell's points
    psi: list[list[np.ndarray]]      # psi[l][k]: (n_c, k_c) wavelets on the cell's points
    V: list[list[np.ndarray]]        # V[l][k]: (s_c, s_c) right singular vectors of M
    sing: list[list[np.ndarray]]     # singular values of M
    offset: list[np.ndarray]         # offset[l][k]: first row of the cell's wavelets in W

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def nwav(self) -> int:
        return self.N - self.p

    def wavelets_of(self, l: int, k: int) -> int:
        return self.psi[l][k].shape[1]

    def cell_points(self, l: int, k: int) -> np.ndarray:
        """Original indices of the cell's points, in permuted (cell) order."""
        t = self.tree
        return t.perm[t.begin[l][k]:t.end[l][k]]

    # --- the operators W, W^T, L -------------------------------------------------
    def apply_W(self, v: np.ndarray) -> np.ndarray:
        out = np.zeros(self.nwav)
        for l in range(self.tree.t, -1, -1):
            for k in range(self.tree.ncells(l)):
                o = self.offset[l][k]
                ps = self.psi[l][k]
                out[o:o + ps.shape[1]] = ps.T @ v[self.cell_points(l, k)]
        return out

    def apply_Wt(self, u: np.ndarray) -> np.ndarray:
        out = np.zeros(self.N)
        for l in range(self.tree.t, -1, -1):
            for k in range(self.tree.ncells(l)):
                o = self.offset[l][k]
                ps = self.psi[l][k]
                out[self.cell_points(l, k)] += ps @ u[o:o + ps.shape[1]]
        return out

    def dense_W(self) -> np.ndarray:
        Wd = np.zeros((self.nwav, self.N))
        for l in range(self.tree.t, -1, -1):
            for k in range(self.tree.ncells(l)):
                o = self.offset[l][k]
                ps = self.psi[l][k]
                Wd[o:o + ps.shape[1], self.cell_points(l, k)] = ps.T
        return Wd

    def dense_L(self) -> np.ndarray:
        Ld = np.zeros((self.p, self.N))
        Ld[:, self.cell_points(0, 0)] = self.phi[0][0].T
        return Ld

    def level_of_row(self) -> np.ndarray:
        lev = np.zeros(self.nwav, dtype=np.int64)
        for l in range(self.tree.t + 1):
            for k in range(self.tree.ncells(l)):
                o = self.offset[l][k]
                lev[o:o + self.wavelets_of(l, k)] = l
        return lev


def build_basis(points: np.ndarray, tree: Tree, w: int, rank_rtol: float | None = None) -> Basis:
    lo, hi = box(points)
    X = design_matrix(points, w, lo, hi)
    p = X.shape[1]
    t = tree.t
    phi = [[None] * tree.ncells(l) for l in range(t + 1)]
    psi = [[None] * tree.ncells(l) for l in range(t + 1)]
    V = [[None] * tree.ncells(l) for l in range(t + 1)]
    sing = [[None] * tree.ncells(l) for l in range(t + 1)]
    for l in range(t, -1, -1):
        for k in range(tree.ncells(l)):
            b, e = tree.begin[l][k], tree.end[l][k]
            idx = tree.perm[b:e]
            n = e - b
            if l == t:
                B = np.eye(n)                                  # leaf unit vectors
            else:
                fl, fr = phi[l + 1][2 * k], phi[l + 1][2 * k + 1]
                B = np.zeros((n, fl.shape[1] + fr.shape[1]))   # children's scaling vectors
                nl = fl.shape[0]
                B[:nl, :fl.shape[1]] = fl
                B[nl:, fl.shape[1]:] = fr
            M = X[idx].T @ B                                   # moments, p x s
            s = B.shape[1]
            U, S, Vh = np.linalg.svd(M, full_matrices=True)
            Vc = Vh.T
            rt = rank_rtol if rank_rtol is not None else 10.0 * max(p, s) * 2.0 ** -52
            a = int(np.sum(S > rt * S[0])) if S.size and S[0] > 0 else 0
            phi[l][k] = B @ Vc[:, :a]
            psi[l][k] = B @ Vc[:, a:]
            V[l][k] = Vc
            sing[l][k] = S
    if phi[0][0].shape[1] != p:
        raise RankDeficient(f"design matrix has numerical rank {phi[0][0].shape[1]} < p = {p}")
    offset = [None] * (t + 1)
    o = 0
    for l in range(t, -1, -1):
        offs = np.zeros(tree.ncells(l), dtype=np.int64)
        for k in range(tree.ncells(l)):
            offs[k] = o
            o += psi[l][k].shape[1]
        offset[l] = offs
    assert o == X.shape[0] - p
    return Basis(tree, p, w, X, lo, hi, phi, psi, V, sing, offset)
