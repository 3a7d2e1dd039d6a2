"""Pins of the extended-precision dense BLUP (oracle.dense_mp) used as the
reference of the ill-conditioned accuracy study (Sec. 8.2, Table 5): facts the
BLUP definition fixes independently of how it is solved."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import dense, dense_mp, design

mp = pytest.importorskip("mpmath")


def test_polynomial_data_is_reproduced_by_the_trend():
    """Z = X beta0 lies in the trend space: the BLUP returns beta0 and gamma = 0
    (eq. Spatial:problem).  (The FP64 rounding of X beta0 puts Z a rounding
    away from the trend space; a moderate width keeps that from being
    amplified.)"""
    P = wl.unit_disk_gaussian(1.0, 0.5, N=30, M=8)
    lo, hi = design.box(P.points)
    X = design.design_matrix(P.points, 3, lo, hi)
    beta0 = np.random.default_rng(3).standard_normal(X.shape[1])
    y, b, g, res = dense_mp.dense_blup_mp(P.points, X @ beta0, P.targets, 3, 0.5, dps=60)
    np.testing.assert_allclose(b, beta0, rtol=1e-10, atol=1e-10)
    assert np.abs(g).max() < 1e-10 * np.abs(X @ beta0).max()
    np.testing.assert_allclose(y, design.design_matrix(P.targets, 3, lo, hi) @ beta0, rtol=1e-12, atol=1e-12)


def test_interpolates_the_data_without_nugget():
    P = wl.unit_disk_gaussian(2.0, 3.0, N=30, M=8)
    y, b, g, res = dense_mp.dense_blup_mp(P.points, P.Z, P.points[:10], 3, 3.0, dps=60)
    np.testing.assert_allclose(y, P.Z[:10], rtol=0, atol=1e-14)


def test_agrees_with_the_fp64_formulae_when_well_conditioned():
    P = wl.unit_disk_gaussian(2.0, 0.3, N=40, M=12)
    ref = dense.dense_blup(P.points, P.Z, P.targets, 2, None, 0.3, 1e-8, family="gaussian")
    y, b, g, res = dense_mp.dense_blup_mp(P.points, P.Z, P.targets, 2, 0.3, nugget=1e-8, dps=40)
    np.testing.assert_allclose(y, ref["yhat"], rtol=1e-9)
    np.testing.assert_allclose(b, ref["beta"], rtol=1e-8)


def test_golden_files_cover_every_row():
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    for alpha, theta in wl.TABLE5_ROWS:
        lines = [l for l in open(os.path.join(here, f"table5_a{alpha:g}_t{theta:g}.txt")) if not l.startswith("#")]
        rows = {l.split()[0]: np.array([float(v) for v in l.split()[1:]]) for l in lines}
        assert rows["yhat"].shape == (200,) and rows["beta"].shape == (math.comb(10, 8),)
        assert np.all(np.isfinite(rows["yhat"]))
