"""The arithmetic of the tensor-core distance tile, modelled on the CPU.

The kernel writes r^2 = |x' - y'' + D|^2 as one contraction over K:
  -2 x'.y''  with every FP32 coordinate split into three BF16 parts
             (h + m + l = the value exactly) and the six products
             h.h, h.m, m.h, h.l, l.h, m.m kept;
  |x'|^2, |y''|^2, R = 2 x'.D + |D|^2 and Q = -2 y''.D, each split in three
             and multiplied by ones;
accumulated in FP32 (every BF16 x BF16 product is exact in FP32).  This
model checks the two facts the design rests on: the split is exact, and the
contraction gives r^2 to about FP32 accuracy relative to the size of the
terms (the offsets from the tile's reference points), while the classic
global-coordinate form loses that accuracy for near pairs."""
import numpy as np


def bf16(v):
    """Round FP32 values to BF16 (8 significant bits), ties to even."""
    v = np.asarray(v, dtype=np.float32)
    b = v.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def split3(v):
    v = np.asarray(v, dtype=np.float32)
    h = bf16(v)
    r1 = (v - h).astype(np.float32)
    m = bf16(r1)
    r2 = (r1 - m).astype(np.float32)
    l = bf16(r2)
    return h, m, l


def test_split_is_exact():
    rng = np.random.default_rng(0)
    for scale in (1e-6, 1e-2, 1.0, 3.7e3):
        v = (rng.standard_normal(20000) * scale).astype(np.float32)
        h, m, l = split3(v)
        assert np.all((h.astype(np.float64) + m + l) == v.astype(np.float64))


def fp32_sum(terms):
    """Sequential FP32 accumulation of exact products (the accumulator)."""
    acc = np.float32(0.0)
    for t in terms:
        acc = np.float32(acc + np.float32(t))
    return float(acc)


def tile_r2(xp, yp, dl):
    """r^2 as the tile's K columns compute it (x' target offset, y'' source
    offset, dl = c_T - c_S), FP32 accumulation in K order."""
    xs = [split3(c) for c in xp]
    ys = [split3(c) for c in yp]
    terms = []
    for (xh, xm, xl), (yh, ym, yl) in zip(xs, ys):          # -2 x'.y'': six products per axis
        for a, b in ((xh, yh), (xh, ym), (xm, yh), (xh, yl), (xl, yh), (xm, ym)):
            terms.append(-2.0 * float(a) * float(b))
    n2x = np.float32(sum(np.float32(c) * np.float32(c) for c in xp))
    n2y = np.float32(sum(np.float32(c) * np.float32(c) for c in yp))
    R = np.float32(2.0 * np.float32(sum(np.float32(a) * np.float32(b) for a, b in zip(xp, dl)))
                   + sum(np.float32(c) * np.float32(c) for c in dl))
    Q = np.float32(-2.0 * np.float32(sum(np.float32(a) * np.float32(b) for a, b in zip(yp, dl))))
    for v in (n2x, n2y, R, Q):
        terms.extend(float(p) for p in split3(v))
    return fp32_sum(terms)


def test_tile_r2_accuracy_for_near_pairs():
    rng = np.random.default_rng(1)
    d = 10
    worst_tile, worst_global = 0.0, 0.0
    for _ in range(300):
        cT = rng.uniform(0, 1, d)
        cS = cT + rng.normal(0, 0.05, d)                   # neighbouring leaves
        x = cT + rng.normal(0, 0.03, d)
        y = x + rng.normal(0, 1e-3, d)                     # a near pair
        x32, y32 = x.astype(np.float32), y.astype(np.float32)
        cT32, cS32 = cT.astype(np.float32), cS.astype(np.float32)
        xp = (x32 - cT32).astype(np.float32)
        yp = (y32 - cS32).astype(np.float32)
        dl = (cT32 - cS32).astype(np.float32)
        exact = float(np.sum((x32.astype(np.float64) - y32.astype(np.float64)) ** 2))
        got = tile_r2(xp, yp, dl)
        scale = float(np.sum(xp.astype(np.float64) ** 2) + np.sum(yp.astype(np.float64) ** 2)
                      + np.sum(dl.astype(np.float64) ** 2))
        worst_tile = max(worst_tile, abs(got - exact) / scale)
        # the classic form on global coordinates, FP32: |x|^2 + |y|^2 - 2 x.y
        g = np.float32(np.sum(x32 * x32) + np.sum(y32 * y32) - np.float32(2) * np.sum(x32 * y32))
        worst_global = max(worst_global, abs(float(g) - exact) / scale)
    # offsets keep the error at FP32 level relative to the offsets' size
    assert worst_tile < 5e-6
    # global coordinates: the same error relative to |x|^2 ~ d/3 is far larger here
    assert worst_global > 10 * worst_tile
