"""Pins of the kd-tree (Algs. 1-3) and the multilevel basis (Sec. 3.1)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import basis as ob, design, tree as ot


def two_pass_var(v):
    m = sum(v) / len(v)
    return sum((a - m) ** 2 for a in v) / len(v)


@pytest.mark.parametrize("N,d,n0", [(1000, 2, 64), (777, 3, 16), (64, 2, 64), (65, 2, 64), (300, 5, 7)])
def test_tree_structure(N, d, n0):
    x = np.random.default_rng(N).random((N, d))
    T = ot.build_tree(x, n0)
    assert sorted(T.perm.tolist()) == list(range(N))
    assert T.t == max(0, math.ceil(math.log2(N / n0))) if N > n0 else T.t == 0
    for l in range(T.t + 1):
        sizes = T.end[l] - T.begin[l]
        assert set(sizes.tolist()) <= {N // 2 ** l, -(-N // 2 ** l)}
        assert T.begin[l][0] == 0 and T.end[l][-1] == N
        assert np.all(T.begin[l][1:] == T.end[l][:-1])
    assert np.all(T.end[T.t] - T.begin[T.t] <= n0)
    if T.t > 0:
        assert np.any(T.end[T.t - 1] - T.begin[T.t - 1] > n0)


def test_rule_max_variance_median_split():
    x = np.random.default_rng(5).random((400, 3)) * np.array([1.0, 3.0, 0.5])
    T = ot.build_tree(x, 20)
    for l in range(T.t):
        for k in range(T.ncells(l)):
            b, e = T.begin[l][k], T.end[l][k]
            pts = x[T.perm[b:e]]
            var = [two_pass_var(list(pts[:, a])) for a in range(3)]
            assert T.axis[l][k] == int(np.argmax(var))
            a = T.axis[l][k]
            h = (e - b) // 2
            left, right = pts[:h, a], pts[h:, a]
            assert left.max() <= T.thr[l][k] < right.min()
            assert len(left) == (e - b) // 2
            # children ranges are the two halves
            assert T.begin[l + 1][2 * k] == b and T.end[l + 1][2 * k + 1] == e
    assert T.axis[0][0] == 1       # the widest axis splits first


def test_tree_boxes():
    x = np.random.default_rng(6).random((200, 2))
    T = ot.build_tree(x, 10)
    for l in range(T.t + 1):
        for k in range(T.ncells(l)):
            pts = x[T.perm[T.begin[l][k]:T.end[l][k]]]
            assert np.all(T.lo[l][k] == pts.min(0)) and np.all(T.hi[l][k] == pts.max(0))


CASES = [(300, 2, 1, 16), (257, 3, 2, 16), (200, 2, 2, 8), (150, 5, 1, 12), (128, 1, 3, 5)]


@pytest.mark.parametrize("N,d,w,n0", CASES)
def test_basis_invariants(N, d, w, n0):
    x = np.random.default_rng(N + d).random((N, d))
    B = ob.build_basis(x, ot.build_tree(x, n0), w)
    p = math.comb(d + w, w)
    W, L = B.dense_W(), B.dense_L()
    assert W.shape == (N - p, N)                                # dim of W (Sec. 3.1)
    np.testing.assert_allclose(W @ B.X, 0, atol=1e-12)          # eq. hbconstruction:eqn1
    np.testing.assert_allclose(W @ W.T, np.eye(N - p), atol=1e-12)
    P = np.vstack([W, L])
    np.testing.assert_allclose(P @ P.T, np.eye(N), atol=1e-12)  # [W; L] orthonormal
    proj = np.eye(N) - B.X @ np.linalg.solve(B.X.T @ B.X, B.X.T)
    np.testing.assert_allclose(W.T @ W, proj, atol=1e-11)       # unique projector onto P^perp
    np.testing.assert_allclose(L.T @ L, np.eye(N) - proj, atol=1e-11)
    v = np.random.default_rng(1).random(N)
    np.testing.assert_allclose(B.apply_W(v), W @ v, atol=1e-13)
    u = np.random.default_rng(2).random(N - p)
    np.testing.assert_allclose(B.apply_Wt(u), W.T @ u, atol=1e-13)


def test_lemma_counts_when_n0_below_2p():
    """Lemmas 1-2 (Sec. 3.1): with n0 < 2p, level q has at most p 2^q wavelets,
    each supported on at most 2^(t-q+1) p points."""
    d, w = 3, 2
    p = math.comb(d + w, w)
    n0 = 2 * p - 1
    x = np.random.default_rng(3).random((600, d))
    T = ot.build_tree(x, n0)
    B = ob.build_basis(x, T, w)
    for q in range(T.t + 1):
        nq = sum(B.wavelets_of(q, k) for k in range(T.ncells(q)))
        assert nq <= p * 2 ** q
        for k in range(T.ncells(q)):
            ps = B.psi[q][k]
            if ps.shape[1]:
                support = np.sum(np.any(np.abs(ps) > 0, axis=1))
                assert support <= 2 ** (T.t - q + 1) * p


def test_direct_sum_dimensions():
    """R^N = P + W_0 + ... + W_t: the level dimensions add up to N - p."""
    x = np.random.default_rng(4).random((500, 2))
    B = ob.build_basis(x, ot.build_tree(x, 20), 2)
    total = sum(B.wavelets_of(l, k) for l in range(B.tree.t + 1) for k in range(B.tree.ncells(l)))
    assert total == 500 - 6
    assert np.all(np.diff(B.level_of_row()) <= 0)     # W = [W_t; ...; W_0]


def test_rank_deficient_design_raises():
    x = np.zeros((50, 2))
    x[:, 0] = np.linspace(0, 1, 50)             # points on a line: x2 monomials vanish
    with pytest.raises(ob.RankDeficient):
        ob.build_basis(x, ot.build_tree(x, 8), 1)


def test_workload_trend_lies_in_design_span():
    P = wl.small_problem(3, 200, 3, 2, nugget=0.0)
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, 2, lo, hi)
    trend = wl._trend(P.points, 2, P.meta["trend_coef"])
    coef, res, *_ = np.linalg.lstsq(X, trend, rcond=None)
    np.testing.assert_allclose(X @ coef, trend, atol=1e-10)
