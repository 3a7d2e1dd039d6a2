"""mlb_apply_W_noalloc: W v computed with a fixed device work space instead of
allocations, for callers that cannot allocate at that moment (graph capture,
allocation-free loops).  Collected last on purpose: a failure here leaves every
other test already run.  Checked against mlb_apply_W on two calls in a row,
which share the work space."""
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
