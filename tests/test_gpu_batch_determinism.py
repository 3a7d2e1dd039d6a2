"""Repeated batched solves must agree bit for bit.

mlb_batch_solve builds its problems' contexts on many host threads at once,
each on its own stream, and runs their PCGs in one persistent launch.  Every
reduction has a fixed order, so any difference between two calls on the same
data can only come from one problem's work reaching another's memory (a
buffer freed while queued kernels still write it, an unordered copy).  The
test repeats one batch and compares statuses, predictions, trend
coefficients and iteration counts exactly."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1701_00285_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_repeats_bit_identical(pkg, prec):
    from paper_1701_00285_gb300.binding import batch_solve, lib
    probs = [q for q in wl.batched_problems(count=120, M=64) if q.N <= 2500][:48]
    assert len(probs) == 48
    items = [{"points": q.points, "w": q.w, "nu": q.nu, "rho": q.rho, "nugget": q.nugget,
              "tau_factor": q.tau_factor, "Z": q.Z, "targets": q.targets} for q in probs]
    first = None
    for call in range(5):
        res, ms, st = batch_solve(items, precision=prec, pcg_rtol=1e-10, pcg_maxit=50000, host_threads=16)
        assert st == 0, lib().mlb_batch_last_error().decode()
        assert all(r[2] == 0 for r in res)
        if first is None:
            first = res
            continue
        for k, (a, b) in enumerate(zip(first, res)):
            assert a[3] == b[3], f"call {call}, problem {k}: iterations {a[3]} vs {b[3]}"
            assert np.array_equal(a[0], b[0]), f"call {call}, problem {k}: predictions differ"
            assert np.array_equal(a[1], b[1]), f"call {call}, problem {k}: trend differs"
