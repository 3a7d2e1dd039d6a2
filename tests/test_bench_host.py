"""Host logic of bench.py (CPU): the roofline bookkeeping and the workload
choices.  Nothing here touches a GPU."""
import hashlib
import json
import math
import os

import bench
import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOLVE = os.path.join(ROOT, "paper_1701_00285_gb300", "csrc", "solve.cu")


def test_kernel_source_extracts_one_function():
    src = bench.kernel_source(SOLVE, "spmv_panel_f32_kernel")
    assert src.startswith("__global__") and src.endswith("}")
    assert "spmv_panel_f32_kernel(" in src and "spmv_panel_f64_kernel(" not in src
    assert bench.kernel_source(SOLVE, "no_such_kernel") == ""


def test_recorded_traffic_is_keyed_to_the_kernel_text(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["spmv_panel_f32_kernel"]
    sha = hashlib.sha256(bench.kernel_source(SOLVE, "spmv_panel_f32_kernel").encode()).hexdigest()[:16]
    got = bench.recorded_traffic("spmv_panel_f32_kernel")
    # the record stands exactly when the committed kernel text is the profiled one
    assert (got == rec["bytes_per_launch"]) == (sha == rec["sha"])
    # a record for another source text is not reported
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / "traffic.json").write_text(json.dumps({"spmv_panel_f32_kernel": dict(rec, sha="0" * 16)}))
    (tmp_path / "paper_1701_00285_gb300").symlink_to(os.path.join(ROOT, "paper_1701_00285_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("spmv_panel_f32_kernel") is None
    assert bench.recorded_traffic("unknown_kernel") is None


def test_matrix_free_choice_and_flop_count():
    assert bench.matrix_free(wl.uniform_10d(N=512, M=8))        # leaf 128, 2p = 132
    assert not bench.matrix_free(wl.heldout_5d(N=512, M=8))     # leaf 64, 2p = 12
    assert bench.ksum_flops_per_pair(10) == 40


def test_describe_names_the_workload_and_its_sizes():
    P = wl.heldout_5d(N=1024, M=16)
    s = bench.describe(P)
    assert s.startswith("heldout_5d_n1024") and "d=5" in s and "16 targets" in s
    assert "tau=inf" in s and math.isinf(P.tau_factor)


def test_power_law_fit_recovers_exponent():
    sizes = [512, 1024, 2048, 4096]
    a, k = bench.fit_power_law(sizes, [3e-9 * n ** 2.6 for n in sizes])
    assert abs(k - 2.6) < 1e-12 and abs(a / 3e-9 - 1) < 1e-9


def test_cpu_baseline_pool_on_a_tiny_sample():
    """Two single-threaded oracle processes on tiny subsamples: the result
    carries the cores used, the per-size medians and iterations, and the
    throughput the fit implies for the full workload."""
    P = wl.heldout_5d(N=4096, M=64)
    P.meta["generator"] = "heldout_5d"
    r = bench.cpu_baseline(P, sizes=(128, 256, 384), workers=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == "BLUP solves/s"
    assert len(r["seconds"]) == 3 and all(t > 0 for t in r["seconds"])
    assert all(i > 0 for i in r["iterations"])
    a, k = bench.fit_power_law(r["sizes"], r["seconds"])
    assert math.isclose(r["value"], 2 / (a * 4096 ** k), rel_tol=1e-12)
