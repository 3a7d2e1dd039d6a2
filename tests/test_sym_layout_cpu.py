"""The symmetric packed storage and its chunked product, modelled on the CPU.

The mixed path stores each symmetric pair of C~_W once: 128-row blocks, each
from its own diagonal square to the right edge (width rounded up to 64,
zero padded), cut into 64-column tiles stored one after the other.  A product
chunk is (block b, column segment s): its rows' sums over the segment go to
rowpart[s][r]; for columns right of the block's diagonal square, its
columns' sums over the block's rows go to colpart[b][c].  q_r is then the
row pieces of r's block followed by the column pieces of the blocks above
it.  This model checks that the layout and the decomposition cover every
(row, column) pair of the full matrix exactly once, for several sizes and
segment widths, including the ragged edges (no GPU needed)."""
import numpy as np
import pytest

ROWS, TILE = 128, 64


def sym_width(n, b):
    return ((n - b * ROWS) + TILE - 1) // TILE * TILE


def pack(A):
    """Blocks of tiles: tile t of block b holds rows x 64 values, row-major."""
    n = A.shape[0]
    nblk = (n + ROWS - 1) // ROWS
    store, off = [], []
    pos = 0
    for b in range(nblk):
        r0, rows, W = b * ROWS, min(ROWS, n - b * ROWS), sym_width(n, b)
        off.append(pos)
        for t in range(W // TILE):
            tile = np.zeros((rows, TILE))
            c0 = r0 + t * TILE
            c1 = min(n, c0 + TILE)
            if c1 > c0:
                tile[:, : c1 - c0] = A[r0:r0 + rows, c0:c1]
            store.append(tile.ravel())
            pos += rows * TILE
    return np.concatenate(store), off, nblk


def chunked_product(vals, off, nblk, n, p, seg):
    rowpart = {}
    colpart = np.zeros((nblk, n))
    for b in range(nblk):
        r0, rows, W = b * ROWS, min(ROWS, n - b * ROWS), sym_width(n, b)
        for s in range(-(-W // seg)):
            cs, ce = r0 + s * seg, min(r0 + W, r0 + (s + 1) * seg)
            rp = np.zeros(rows)
            for c0 in range(cs, ce, TILE):
                t = (c0 - r0) // TILE
                tile = vals[off[b] + t * rows * TILE: off[b] + (t + 1) * rows * TILE].reshape(rows, TILE)
                cols = np.arange(c0, c0 + TILE)
                pc = np.where(cols < n, p[np.minimum(cols, n - 1)], 0.0)
                rp += tile @ pc
                right = (cols >= r0 + ROWS) & (cols < n)
                colpart[b, cols[right]] = (tile.T @ p[r0:r0 + rows])[right]
            rowpart[(b, s)] = rp
    q = np.zeros(n)
    for r in range(n):
        b = r // ROWS
        ns = -(-sym_width(n, b) // seg)
        acc = 0.0
        for s in range(ns):
            acc += rowpart[(b, s)][r - b * ROWS]
        for bb in range(b):
            acc += colpart[bb, r]
        q[r] = acc
    return q


@pytest.mark.parametrize("n", [1, 37, 128, 129, 300, 517])
@pytest.mark.parametrize("seg", [256, 512])
def test_chunked_symmetric_product_covers_every_pair_once(n, seg):
    rng = np.random.default_rng(n * 7 + seg)
    B = rng.standard_normal((n, n))
    A = B + B.T
    p = rng.standard_normal(n)
    vals, off, nblk = pack(A)
    q = chunked_product(vals, off, nblk, n, p, seg)
    np.testing.assert_allclose(q, A @ p, rtol=1e-12, atol=1e-12 * np.abs(A).sum(axis=1).max())


def test_packed_storage_holds_each_pair_once_plus_the_squares():
    """Stored values: every block's rows over its width, which is the upper
    triangle by blocks plus the full diagonal squares and the padding."""
    n = 300
    A = np.arange(n * n, dtype=float).reshape(n, n)
    A = A + A.T
    vals, off, nblk = pack(A)
    expect = sum(min(ROWS, n - b * ROWS) * sym_width(n, b) for b in range(nblk))
    assert vals.size == expect
    assert expect < n * n                      # fewer than both triangles
