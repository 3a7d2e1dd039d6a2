"""Pins of the distance criterion and tree search (Sec. 4.1, Algs. 4-6)."""
import math

import numpy as np
import pytest

from oracle import pattern as op, tree as ot


@pytest.mark.parametrize("c", [0.0, 0.3, 1.0, 2.0, math.inf])
@pytest.mark.parametrize("seed,N,d,n0", [(0, 400, 2, 16), (1, 300, 3, 10), (2, 256, 5, 16)])
def test_search_equals_bruteforce(c, seed, N, d, n0):
    x = np.random.default_rng(seed).random((N, d))
    T = ot.build_tree(x, n0)
    ps, pb = op.pattern(T, c, "search"), op.pattern(T, c, "brute")
    for key in pb:
        assert np.array_equal(ps[key], pb[key]), key
    for l in range(T.t + 1):
        assert np.array_equal(pb[(l, l)], pb[(l, l)].T)          # symmetric within a level
        assert np.all(np.diag(pb[(l, l)]))                       # a cell meets itself
    if math.isinf(c):
        assert all(v.all() for v in pb.values())


def test_tree_search_reaches_every_box_meeting_cell():
    """The kd-region search (no box filter) returns a superset of the box test."""
    x = np.random.default_rng(7).random((500, 2))
    T = ot.build_tree(x, 16)
    for i in range(T.t + 1):
        for j in range(i, T.t + 1):
            brute = op.level_pair_bruteforce(T, i, j, 1.0)
            tau = op.tau_levels(T, i, j, 1.0)
            for m in range(T.ncells(i)):
                found = set(op.search_tree(T, T.lo[i][m], T.hi[i][m], j, tau))
                assert set(np.nonzero(brute[m])[0]) <= found


def test_hand_example_one_dimension():
    """Eight points on a line, leaves of 2: cells {0,1},{2,3},{4,5},{6,7} at
    positions 0, .1 | .2, .3 | 1, 1.1 | 3, 3.1.  Leaf diameters 0.1, mean 0.1;
    with c = 2, tau_22 = 0.2, so leaf 0 meets leaf 1 (gap 0.1) but not leaf 2
    (gap 0.7).  Level-1 cells [0, .3] and [1, 3.1] have diameters .3 and 2.1,
    mean 1.2, so tau_11 = 2.4 and tau_12 = 2 sqrt(1.2 * 0.1) = 0.6928."""
    x = np.array([0.0, 0.1, 0.2, 0.3, 1.0, 1.1, 3.0, 3.1])[:, None]
    T = ot.build_tree(x, 2)
    assert T.t == 2
    adm = op.level_pair_bruteforce(T, 2, 2, 2.0)
    expect = np.array([[1, 1, 0, 0], [1, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], bool)
    assert np.array_equal(adm, expect)
    assert op.level_pair_bruteforce(T, 1, 1, 2.0).all()            # gap .7 < 2.4
    # cross level: [0, .3] misses [1, 1.1] (gap .7 > .6928) and [3, 3.1];
    # [1, 3.1] misses [0, .1] (gap .9) and [.2, .3] (gap .7)
    cross = op.level_pair_bruteforce(T, 1, 2, 2.0)
    assert np.array_equal(cross, np.array([[1, 1, 0, 0], [0, 0, 1, 1]], bool))
    assert abs(op.tau_levels(T, 1, 2, 2.0) - 2 * math.sqrt(1.2 * 0.1)) < 1e-15
