"""mlb_apply_W_noalloc: W v computed with a fixed device work space instead of
allocations, for callers that cannot allocate at that moment (loops that must
not block on the allocator, a fixed device-memory budget, memory owned by
another framework's pool).  Collected last on purpose: a failure here leaves
every other test already run.  Checked against mlb_apply_W on two calls in a
row, which share the work space, and at the exact size limit."""
import math

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_transform_matches_apply_W_on_consecutive_calls():
    import torch
    import paper_1701_00285_gb300 as pkg

    P = wl.small_problem(900, 3000, 3, 2, leaf_size=32)
    ctx = pkg.Context("fp64", leaf_size=32)
    ctx.build_basis(P.points, 2)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    rng = np.random.default_rng(11)
    for call in range(2):
        v = rng.standard_normal(P.N)
        expect = ctx.apply_W(v)
        v_dev = torch.from_numpy(v).cuda()
        out = torch.full((ctx.nwav,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ctx.apply_W_noalloc(v_dev.data_ptr(), out.data_ptr())
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-12)


def test_noalloc_transform_rejects_sizes_beyond_its_work_space():
    import torch
    import paper_1701_00285_gb300 as pkg

    x = np.random.default_rng(12).random((600000, 2))
    ctx = pkg.Context("fp64", leaf_size=64)
    ctx.build_basis(x, 1)
    v = torch.zeros(600000, dtype=torch.float64, device="cuda")
    out = torch.zeros(ctx.nwav, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.MLBError) as e:
        ctx.apply_W_noalloc(v.data_ptr(), out.data_ptr())
    assert e.value.name == "EINVAL" and "work space" in str(e.value)


def test_noalloc_transform_at_the_exact_size_limit():
    """d = 2, w = 1 (p = 3), leaf 64: every one of the 2^14 - 1 cells of a
    depth-13 tree keeps 3 scaling coefficients, so N = 524,288 - 3 (2^14 - 1)
    fills the work space exactly and one more point exceeds it."""
    import torch
    import paper_1701_00285_gb300 as pkg

    n_fit = 524288 - 3 * (2 ** 14 - 1)
    x = np.random.default_rng(13).random((n_fit + 1, 2))
    for n, ok in ((n_fit, True), (n_fit + 1, False)):
        ctx = pkg.Context("fp64", leaf_size=64)
        ctx.build_basis(x[:n], 1)
        assert ctx.t == 13
        v = np.random.default_rng(14).standard_normal(n)
        v_dev = torch.from_numpy(v).cuda()
        out = torch.full((ctx.nwav,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if ok:
            ctx.apply_W_noalloc(v_dev.data_ptr(), out.data_ptr())
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), ctx.apply_W(v), rtol=1e-12, atol=1e-12)
        else:
            with pytest.raises(pkg.MLBError) as e:
                ctx.apply_W_noalloc(v_dev.data_ptr(), out.data_ptr())
            assert e.value.name == "EINVAL"
        ctx.close()
