"""Sparse multilevel covariance C~_W (Sec. 4, Algorithm 7).

For every level pair (i, j >= i), every source cell B^i_m and every target cell
B^j_q found by the distance criterion, every wavelet pair gives the entry
(psi^i_k)^T C psi^j_l.  The block of the pair is Psi_m^T C(S_m, S_q) Psi_q with
C(S_m, S_q) the covariance between the two cells' points (kernel values plus
the nugget where the two points coincide).  Blocks with j > i are mirrored
(Remark after Algorithm 6); blocks of one level are computed for every
admissible ordered pair, which is symmetric by construction of the pattern.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import Basis
from .matern import kernel_matrix
from .pattern import pattern as make_pattern


def cell_cov(basis: Basis, points: np.ndarray, li: int, m: int, lj: int, q: int,
             nu: float, rho: float, nugget: float, **kf) -> np.ndarray:
    im, iq = basis.cell_points(li, m), basis.cell_points(lj, q)
    C = kernel_matrix(points[im], points[iq], nu, rho, **kf)
    if nugget:
        same = im[:, None] == iq[None, :]
        C = C + nugget * same
    return C


def block(basis: Basis, points, li, m, lj, q, nu, rho, nugget, **kf) -> np.ndarray:
    """Psi_m^T C(S_m, S_q) Psi_q for cell m of level li and q of level lj."""
    C = cell_cov(basis, points, li, m, lj, q, nu, rho, nugget, **kf)
    return basis.psi[li][m].T @ C @ basis.psi[lj][q]


def assemble(basis: Basis, points: np.ndarray, nu: float, rho: float, nugget: float,
             tau_factor: float, pat=None, **kf) -> dict:
    """Algorithm 7 over all level pairs.  Returns {(li, m, lj, q): block} holding
    both (m, q) and the mirrored (q, m) entries, plus the pattern."""
    if pat is None:
        pat = make_pattern(basis.tree, tau_factor)
    blocks = {}
    for (i, j), adm in pat.items():
        for m in range(adm.shape[0]):
            if basis.wavelets_of(i, m) == 0:
                continue
            for q in np.nonzero(adm[m])[0]:
                if basis.wavelets_of(j, q) == 0:
                    continue
                if i == j and q < m:
                    continue
                B = block(basis, points, i, m, j, int(q), nu, rho, nugget, **kf)
                blocks[(i, m, j, int(q))] = B
                if (i, m) != (j, int(q)):
                    blocks[(j, int(q), i, m)] = B.T
    return {"blocks": blocks, "pattern": pat}


def to_sparse(basis: Basis, asm: dict) -> sp.csr_matrix:
    rows, cols, vals = [], [], []
    for (i, m, j, q), B in asm["blocks"].items():
        om, oq = basis.offset[i][m], basis.offset[j][q]
        r = om + np.arange(B.shape[0])
        c = oq + np.arange(B.shape[1])
        rr, cc = np.meshgrid(r, c, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(B.ravel())
    n = basis.nwav
    if not rows:
        return sp.csr_matrix((n, n))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def block_norms(basis: Basis, asm: dict) -> dict:
    """Frobenius norm of every stored block: invariant under the choice of
    orthonormal wavelets inside each cell (SVD sign/rotation freedom)."""
    return {key: float(np.linalg.norm(B)) for key, B in asm["blocks"].items()}
