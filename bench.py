#!/usr/bin/env python
"""Benchmark of the multilevel BLUP hot path on one GB300 (or N replicas).

One step = one BLUP solve from scratch on the resident inputs: kd-tree and
multilevel basis, assembly of C~_W, diagonal PCG, gamma = W^T gamma_W, the
trend step and the prediction at the targets (every row of the hot path).

Workload (default): n = 32,768 points uniform in [0,1]^5, Matern nu = 3/2,
rho = 0.3, nugget 1e-4, w = 1 (p = 6), leaf size 64, tau = inf (the full
C_W, 1.07e9 entries), PCG tol 1e-10, 4,096 held-out targets.  Synthetic,
seeded.  `--workload clustered_3d` (n = 65,536 in [0,1]^3 with 8 tight
clusters, nugget 1e-6, tau = 2 diameters), `uniform_10d` (d = 10,
matrix-free) and `batched_problems` are available too.

Prints one JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 1.25    # GB300 dense FP64, nominal (152 SMs at 2.07 GHz)
FP32_PEAK_TFLOPS = 80.5    # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
METRIC = "BLUP solves/s & C_W entries/s, mixed vs FP64 GPU at 1e-5 rel err; % roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--single", action="store_true", help="measure only --precision")
    ap.add_argument("--workload", default="heldout_5d",
                    choices=["heldout_5d", "clustered_3d", "uniform_10d", "batched_problems"])
    ap.add_argument("--count", type=int, default=64,
                    help="batched_problems: number of problems (the full workload is 512; 64 keeps both precisions "
                         "with 3 + 3 steps within minutes)")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--targets", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra keys: full-size clustered_3d assembly and uniform_10d product")
    ap.add_argument("--mse", type=int, default=0,
                    help="time the kriging MSE at this many targets instead (one PCG solve each)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks -----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- helpers -----
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            j = json.load(f)
        return j.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_source(path: str, kernel: str) -> str:
    """Text of one __global__ function: from its declaration to the first line
    that closes it (a lone "}" at column 0)."""
    lines = open(path).read().splitlines()
    for i, line in enumerate(lines):
        if "__global__" in line and f" {kernel}(" in line:
            for k in range(i, len(lines)):
                if lines[k] == "}":
                    return "\n".join(lines[i:k + 1])
    return ""


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of the kernel (sha256 of the function's text)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        j = json.load(f).get(kernel)
    if not j:
        return None
    src = kernel_source(os.path.join(ROOT, "paper_1701_00285_gb300", "csrc", j["file"]), kernel)
    sha = hashlib.sha256(src.encode()).hexdigest()[:16]
    return j["bytes_per_launch"] if src and sha == j["sha"] else None


def workload(args, rank=0):
    import workloads as wl
    kw = {}
    if args.n:
        kw["N"] = args.n
    if args.targets:
        kw["M"] = args.targets
    P = getattr(wl, args.workload)(**kw)
    P.meta["generator"] = args.workload     # lets the oracle sample draw the same workload
    return P


def matrix_free(P) -> bool:
    return P.leaf_size > 64 or 2 * math.comb(P.d + P.w, P.w) > 64


def ksum_flops_per_pair(d: int) -> int:
    """Algorithmic FP32 work of one kernel-sum pair: d differences and d
    multiply-adds (3d flops), square root, scaling, exponential, Matern
    polynomial and the weighted accumulation (10)."""
    return 3 * d + 10


def describe(P) -> str:
    tau = "inf (full C_W)" if math.isinf(P.tau_factor) else f"{P.tau_factor:g} cell diameters"
    return (f"{P.name}: multilevel BLUP, n={P.N}, d={P.d}, Matern nu={P.nu:g} rho={P.rho:g} "
            f"nugget={P.nugget:g}, w={P.w} (p={math.comb(P.d + P.w, P.w)}), leaf {P.leaf_size}, "
            f"tau={tau}, PCG tol {P.pcg_rtol:g}, {P.targets.shape[0]} targets")


ORACLE_SIZES = (512, 1024, 2048)


def _oracle_worker(name: str, sizes, seed: int, n: int, m: int):
    """One single-threaded oracle process: the multilevel BLUP (Alg. 7
    assembly, PCG, trend step, prediction) on a seeded subsample of the
    workload at each size, targets in the workload's proportion.  Returns
    [(size, seconds, PCG iterations)]."""
    import workloads as wl
    from oracle import mlblup
    P = getattr(wl, name)(N=n, M=m)
    out = []
    for s in sizes:
        S = wl.subsample(P, s, seed=seed, m=max(1, s * m // n))
        t0 = time.perf_counter()
        r = mlblup.blup(S.points, S.Z, S.targets, S.w, S.nu, S.rho, S.nugget, S.leaf_size,
                        tau_factor=S.tau_factor, rtol=S.pcg_rtol, maxit=20000)
        out.append((s, time.perf_counter() - t0, int(r["info"].get("iterations", 0))))
    return out


def fit_power_law(sizes, seconds):
    """Least-squares fit of log t = log a + k log n; returns (a, k)."""
    x = np.log(np.asarray(sizes, dtype=np.float64))
    y = np.log(np.asarray(seconds, dtype=np.float64))
    k, la = np.polyfit(x, y, 1)
    return float(math.exp(la)), float(k)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(P, sizes=ORACLE_SIZES, workers=None):
    """The oracle as it stands (numpy FP64), timed on every host core: one
    single-threaded process per core (a spawned pool, safe beside an
    initialised CUDA context), all running the same seeded subsamples of the
    workload at once.  The per-size medians are fitted with t = a n^k and the
    fit gives the time of one full-size solve on one loaded core; the cores
    together finish `cores` such solves in that time."""
    import multiprocessing as mp
    C = workers or host_cores()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(C) as pool:
            res = pool.starmap(_oracle_worker, [(P.meta["generator"], tuple(sizes), 1 + k, P.N, P.targets.shape[0])
                                                for k in range(C)])
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    med = [float(np.median([r[i][1] for r in res])) for i in range(len(sizes))]
    its = [int(np.median([r[i][2] for r in res])) for i in range(len(sizes))]
    a, k = fit_power_law(sizes, med)
    t_full = a * P.N ** k
    value = C / t_full
    return {"value": value, "unit": "BLUP solves/s", "cores": C, "kind": "oracle",
            "sample": (f"oracle multilevel BLUP (Alg. 7 assembly, PCG, trend, prediction) on seeded subsamples "
                       f"n = {', '.join(str(s) for s in sizes)} (targets in the workload's proportion), one "
                       f"single-threaded process per host core ({C} at once, {wall:.1f} s wall); median seconds "
                       f"{', '.join(f'{t:.2f}' for t in med)}, PCG iterations {', '.join(str(i) for i in its)}; "
                       f"fit t = {a:.3g} n^{k:.2f} gives {t_full:.0f} s per N={P.N} solve per core"),
            "sizes": list(sizes), "seconds": med, "iterations": its, "exponent": k,
            "seconds_full_size_per_core": t_full, "wall_seconds": wall}


# ------------------------------------------------------------ reference -----
def run_reference(args, rank, world):
    """The oracle arm: every step is one cpu_baseline measurement (all host
    cores, the same procedure as the cpu_baseline key of the GPU arm); the
    value is the median over the timed steps."""
    if rank != 0:
        return
    P = workload(args)
    for _ in range(max(0, args.warmup)):
        cpu_baseline(P, sizes=ORACLE_SIZES[:2])     # two sizes: the fit stays defined
    runs = [cpu_baseline(P) for _ in range(args.steps)]
    value = float(np.median([r["value"] for r in runs]))
    cb = runs[-1]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "BLUP solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * cb["cores"] / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(P), "cache": "oracle on host cores"},
            "cpu_baseline": {"value": value, "unit": "BLUP solves/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"], "exponent": cb["exponent"]},
            "e2e": {"value": value, "unit": "BLUP solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours -----
def measure(pkg, torch, P, precision, args, dev, local_rank, world, stream):
    """Warm-up, then K timed steps of one precision on the resident inputs."""
    N, d, M, p = P.N, P.d, P.targets.shape[0], math.comb(P.d + P.w, P.w)
    # the assembled panels need leaf <= 64 and 2p <= 64; larger cells (the
    # d = 10 workload) take the matrix-free three-step product, P_W = I
    mf = matrix_free(P)
    ctx = pkg.Context(precision, leaf_size=P.leaf_size, pcg_rtol=P.pcg_rtol, pcg_maxit=50000,
                      device=local_rank, matrix_free=mf, precond=not mf)
    ctx.set_stream(stream.cuda_stream)
    with torch.cuda.stream(stream):
        pts = torch.from_numpy(P.points).to(dev)
        Z = torch.from_numpy(P.Z).to(dev)
        tg = torch.from_numpy(P.targets).to(dev)
        yhat = torch.empty(M, dtype=torch.float64, device=dev)
        beta = torch.empty(p, dtype=torch.float64, device=dev)
    stream.synchronize()
    infos = []

    def step():
        ctx.build_basis_dev(pts.data_ptr(), N, d, P.w)
        ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)
        infos.append(ctx.solve_dev(Z.data_ptr(), beta.data_ptr()))
        ctx.predict_dev(tg.data_ptr(), M, yhat.data_ptr())

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    infos.clear()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        e1.synchronize()
    launches = ctx.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    info = infos[-1]
    out = {"ctx": ctx, "ms": ms, "ms_step": ms / args.steps, "value": world * args.steps / (ms / 1000.0),
           "info": info, "launches": launches, "clocks": clk.summary(),
           "yhat": yhat.cpu().numpy(), "beta": beta.cpu().numpy()}

    # build_basis alone (kd-tree, basis, cell tables), so that solves/s can be
    # stated both with and without it
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(3):
        ctx.build_basis_dev(pts.data_ptr(), N, d, P.w)
    b1.record(stream)
    b1.synchronize()
    out["basis_ms"] = b0.elapsed_time(b1) / 3
    ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)    # leave the context assembled

    # the PCG matrix-vector product alone, timed live on its stream
    nwav = N - p
    with torch.cuda.stream(stream):
        u = torch.randn(nwav, dtype=torch.float64, device=dev)
        o = torch.empty(nwav, dtype=torch.float64, device=dev)
    stream.synchronize()
    reps = 20
    for _ in range(3):
        ctx.cw_matvec_dev(u.data_ptr(), o.data_ptr())
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(reps):
        ctx.cw_matvec_dev(u.data_ptr(), o.data_ptr())
    s1.record(stream)
    s1.synchronize()
    out["spmv_ms"] = s0.elapsed_time(s1) / reps
    out["matrix_free"] = mf
    vb = 4 if precision == "mixed" else 8
    if info.get("symmetric"):
        # symmetric storage: the algorithmic bytes of one product are the
        # unique entries (blocks j >= i) once, x read and y written once;
        # the form of the product is the one the library's autotuner kept
        out["spmv_kernel"] = "sym_spmv_bulk_kernel" if info.get("product_variant") == 1 else "sym_spmv_f32_kernel"
        out["spmv_bytes"] = info["nnz_unique"] * 4 + 2 * nwav * 8
    else:
        # row panels: every stored value once, each panel's column list once,
        # x read and y written once
        out["spmv_kernel"] = "spmv_panel_f32_kernel" if precision == "mixed" else "spmv_panel_f64_kernel"
        out["spmv_bytes"] = info["nnz"] * vb + info["col_total"] * 4 + 2 * nwav * 8
    out["matrix_bytes"] = info["product_values"] * vb
    return out


def extra_assembly(pkg, torch, stream, local_rank):
    """The sparse workload's assembly at full size (n = 65,536 in [0,1]^3,
    half in 8 tight clusters, tau = 2 level-mean diameters): C~_W entries/s
    in both precisions, timed with CUDA events on the context's stream (the
    assembly's own device time, mlb_info.ms_assemble).  Its truncated system
    is indefinite, so no solve is timed."""
    import workloads as wl
    P = wl.clustered_3d(M=16)
    out = {"workload": describe(P)}
    for prec in ("mixed", "fp64"):
        ctx = pkg.Context(prec, leaf_size=P.leaf_size, device=local_rank)
        ctx.set_stream(stream.cuda_stream)
        ctx.build_basis(P.points, P.w)
        ms = []
        for _ in range(3):
            ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)
            ms.append(ctx.info()["ms_assemble"])
        inf = ctx.info()
        ctx.close()
        t = statistics.median(ms[1:])
        out[prec] = {"ms_assemble": t, "cw_entries_per_s": inf["nnz_unique"] / (t / 1000.0),
                     "nnz_unique": inf["nnz_unique"], "nnz_stored": inf["nnz"]}
    return out


def extra_matrix_free_product(pkg, torch, stream, local_rank):
    """One full-size product of the high-dimensional workload (n = 262,144 in
    [0,1]^10, nu = 5/2, leaf 128, w = 2): the three-step product W (C (W^T u))
    whose N x N FP32 kernel sum dominates; CUDA events on the stream."""
    import workloads as wl
    P = wl.uniform_10d(M=16)
    ctx = pkg.Context("mixed", leaf_size=P.leaf_size, matrix_free=True, precond=False, device=local_rank)
    ctx.set_stream(stream.cuda_stream)
    ctx.build_basis(P.points, P.w)
    ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)
    with torch.cuda.stream(stream):
        u = torch.randn(ctx.nwav, dtype=torch.float64, device=f"cuda:{local_rank}")
        o = torch.empty_like(u)
    ctx.cw_matvec_dev(u.data_ptr(), o.data_ptr())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        ctx.cw_matvec_dev(u.data_ptr(), o.data_ptr())
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    variant = ctx.info()["product_variant"]     # the autotuner's choice for this size
    ctx.close()
    flops = float(P.N) * P.N * ksum_flops_per_pair(P.d)
    achieved = flops / (ms / 1000.0) / 1e12
    kernel = "ksum_tc_kernel" if variant == 6 else "ksum_f32_kernel"
    return {"workload": describe(P), "ms_per_product": ms, "pairs_per_s": float(P.N) * P.N / (ms / 1000.0),
            "product_variant": variant,
            "roofline": {"kernel": kernel, "bound": "alu", "achieved": achieved,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                         "peak_source": "nominal", "algorithmic_flops": flops}}


def e2e_run(ctx, P, args, world, torch, dev=None):
    hp, hz, ht = P.points.copy(), P.Z.copy(), P.targets.copy()
    ctx.set_stream(None)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.build_basis(hp, P.w)
        ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)
        hb, _ = ctx.solve(hz)
        hy = ctx.predict(ht)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world, dev)
    return {"value": world * args.steps / dt, "unit": "BLUP solves/s",
            "h2d_bytes_per_step": int(hp.nbytes + hz.nbytes + ht.nbytes),
            "d2h_bytes_per_step": int(hy.nbytes + hb.nbytes)}


def shard_indices(count: int, rank: int, world: int) -> range:
    """Problems of one rank: its own slice of the world x count problems the
    generator draws (weak scaling; ranks share nothing)."""
    return range(rank * count, (rank + 1) * count)


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device) -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_batched(args, rank, world, local_rank):
    """Batched workload: every step solves this rank's problems in one
    mlb_batch_solve (host buffers in, predictions out: end to end)."""
    import torch
    import workloads as wl
    from paper_1701_00285_gb300.binding import batch_last_launches, batch_last_phase_ms, batch_solve
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    every = wl.batched_problems(count=args.count * world)
    probs = [every[i] for i in shard_indices(args.count, rank, world)]
    items = [{"points": q.points, "w": q.w, "nu": q.nu, "rho": q.rho, "nugget": q.nugget,
              "tau_factor": q.tau_factor, "Z": q.Z, "targets": q.targets} for q in probs]
    h2d = sum(q.points.nbytes + q.Z.nbytes + q.targets.nbytes for q in probs)
    d2h = sum(q.targets.shape[0] * 8 + math.comb(q.d + q.w, q.w) * 8 for q in probs)
    out = {}
    for prec in ("mixed", "fp64"):
        for _ in range(args.warmup):
            res, ms, st = batch_solve(items, precision=prec, pcg_rtol=1e-10, pcg_maxit=50000, device=local_rank)
        launches = 0
        with ClockSampler(local_rank) as clk:
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                res, ms, st = batch_solve(items, precision=prec, pcg_rtol=1e-10, pcg_maxit=50000, device=local_rank)
                launches += batch_last_launches()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            barrier(world)
        out[prec] = {"res": res, "s": max_over_ranks(dt, world, dev), "status": st, "clocks": clk.summary(),
                     "its": [r[3] for r in res], "phases": batch_last_phase_ms(), "launches": launches}
    ym = np.concatenate([r[0] for r in out["mixed"]["res"]])
    yd = np.concatenate([r[0] for r in out["fp64"]["res"]])
    per = [float(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0])) for a, b in zip(out["mixed"]["res"], out["fp64"]["res"])]
    value = world * args.count * args.steps / out["mixed"]["s"]
    line = {"metric": METRIC, "value": value, "unit": "BLUP solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * out["mixed"]["s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": f"batched_problems: {args.count} independent problems per GPU, n log-uniform [500, 8000], "
                                   f"d in {{2,3,5}}, nu in {{1/2,3/2,5/2}}, rho ~ U[0.1,0.5], w=1, leaf 64, "
                                   f"tau=inf, nugget 1e-4, PCG tol 1e-10, 1024 targets each",
                       "precision": "mixed", "parallelism": f"problem-sharded{world}",
                       "cache": "inputs copied from the host each step (batched API takes host buffers)"},
            "e2e": {"value": value, "unit": "BLUP solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": out["mixed"]["launches"],
            "launches_per_problem": out["mixed"]["launches"] / (args.steps * args.count),
            "phases_ms": out["mixed"]["phases"],
            "fp64": {"value": world * args.count * args.steps / out["fp64"]["s"],
                     "ms_per_step": 1000 * out["fp64"]["s"] / args.steps, "phases_ms": out["fp64"]["phases"]},
            "mixed_vs_fp64": {"rel_pred_err_max": max(per), "rel_pred_err_all": float(np.linalg.norm(ym - yd) / np.linalg.norm(yd)),
                              "speedup": out["fp64"]["s"] / out["mixed"]["s"]},
            "pcg_iterations": {"median": float(np.median(out["mixed"]["its"])), "max": int(max(out["mixed"]["its"]))},
            "status": out["mixed"]["status"], "clocks": out["mixed"]["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_mse(args, rank, world, local_rank):
    """Kriging MSE at K targets of the workload (the formula after eq.
    Spatial): one multilevel PCG solve per target on the assembled C~_W.
    Prints its own JSON line: MSE targets/s per precision."""
    import torch
    import paper_1701_00285_gb300 as pkg
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    P = workload(args, rank)
    K = args.mse
    tg = np.ascontiguousarray(P.targets[:K])
    out = {}
    for prec in ("mixed", "fp64"):
        ctx = pkg.Context(prec, leaf_size=P.leaf_size, pcg_rtol=P.pcg_rtol, pcg_maxit=50000, device=local_rank)
        ctx.build_basis(P.points, P.w)
        ctx.assemble(P.nu, P.rho, P.nugget, P.tau_factor)
        for _ in range(args.warmup):
            ctx.mse(tg[:1])
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = ctx.mse(tg)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        out[prec] = {"value": world * K / dt, "s": dt, "mse": m}
        ctx.close()
    line = {"metric": "kriging MSE at targets (one multilevel PCG solve each)", "value": out["mixed"]["value"],
            "unit": "targets/s", "n_gpus": world, "targets": K, "higher_is_better": True, "scaling": "weak",
            "dtype": "f32/f64", "data": "synthetic", "config": {"workload": describe(P)},
            "fp64": {"value": out["fp64"]["value"]},
            "mixed_vs_fp64_max_abs": float(np.max(np.abs(out["mixed"]["mse"] - out["fp64"]["mse"]))),
            "mse_range": [float(out["fp64"]["mse"].min()), float(out["fp64"]["mse"].max())]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1701_00285_gb300 as pkg

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    P = workload(args, rank)
    stream = torch.cuda.Stream(device=dev)
    head = measure(pkg, torch, P, args.precision, args, dev, local_rank, world, stream)
    other_prec = "fp64" if args.precision == "mixed" else "mixed"
    other = None if args.single else measure(pkg, torch, P, other_prec, args, dev, local_rank, world, stream)
    e2e = None if args.no_e2e else e2e_run(head["ctx"], P, args, world, torch, dev)
    info = head["info"]
    if head["matrix_free"]:
        # three-step product: the N x N kernel sum dominates (the tensor-core
        # form when the autotuner kept it, variant 6)
        kname = "ksum_tc_kernel" if info.get("product_variant") == 6 else "ksum_f32_kernel"
        flops = float(P.N) * P.N * ksum_flops_per_pair(P.d)
        achieved = flops / (head["spmv_ms"] / 1000.0) / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS, "peak_source": "nominal",
                "traffic": None, "algorithmic_flops": flops, "ms_per_launch": head["spmv_ms"]}
    elif args.precision == "mixed":
        # FP32 panels: 4 bytes per entry against HBM bandwidth
        peak, peak_kind = peaks()
        kname = head["spmv_kernel"]
        achieved = head["spmv_bytes"] / (head["spmv_ms"] / 1000.0) / 1e9
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": recorded_traffic(kname),
                "algorithmic_bytes": head["spmv_bytes"], "ms_per_launch": head["spmv_ms"]}
    else:
        # FP64 panels: one FMA per entry; GB300's FP64 rate (nominal 1.25 TFLOP/s)
        # is below what 8 bytes per entry at HBM speed would need
        kname = "spmv_panel_f64_kernel"
        flops = 2.0 * info["nnz"]
        achieved = flops / (head["spmv_ms"] / 1000.0) / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": "nominal",
                "traffic": recorded_traffic(kname), "algorithmic_bytes": head["spmv_bytes"],
                "ms_per_launch": head["spmv_ms"]}
    line = {"metric": METRIC, "value": head["value"], "unit": "BLUP solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": describe(P), "precision": args.precision,
                       "parallelism": f"replicas{world}",
                       "cache": ("matrix-free: compute-bound N^2 kernel sums; inputs (%.0f MB) not flushed"
                                 % (P.points.nbytes / 1e6)) if head["matrix_free"] else
                                ("working set (C~_W %.1f GB%s) larger than L2"
                                 % (head["matrix_bytes"] / 1e9,
                                    ", each symmetric pair once" if info.get("symmetric") else ""))},
            "cw_entries_per_s": info["nnz_unique"] / (info["ms_assemble"] / 1000.0) if info["ms_assemble"] else None,
            "value_without_basis": 1000.0 * world / (head["ms_step"] - head["basis_ms"]),
            "basis_ms": head["basis_ms"],
            "phases_ms": {"assemble": info["ms_assemble"], "pcg": info["ms_pcg"], "trend": info["ms_beta"]},
            "pcg_iterations": info["iterations"], "nnz": info["nnz"], "nnz_unique": info["nnz_unique"],
            "roofline": roof, "e2e": e2e, "gpu_launches": head["launches"], "clocks": head["clocks"]}
    if other is not None:
        oi = other["info"]
        ref, got = (other, head) if args.precision == "mixed" else (head, other)
        line[other_prec] = {"value": other["value"], "ms_per_step": other["ms_step"],
                            "phases_ms": {"assemble": oi["ms_assemble"], "pcg": oi["ms_pcg"], "trend": oi["ms_beta"]},
                            "pcg_iterations": oi["iterations"],
                            "cw_entries_per_s": oi["nnz_unique"] / (oi["ms_assemble"] / 1000.0) if oi["ms_assemble"] else None,
                            "spmv_ms": other.get("spmv_ms"), "clocks": other["clocks"]}
        line["mixed_vs_fp64"] = {
            "rel_pred_err": float(np.linalg.norm(got["yhat"] - ref["yhat"]) / np.linalg.norm(ref["yhat"])),
            "rel_beta_err": float(np.linalg.norm(got["beta"] - ref["beta"]) / np.linalg.norm(ref["beta"])),
            "speedup": (head["value"] / other["value"]) if args.precision == "mixed" else (other["value"] / head["value"])}
        other["ctx"].close()
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "heldout_5d" and args.n is None:
        line["clustered_3d_assembly"] = extra_assembly(pkg, torch, stream, local_rank)
        line["uniform_10d_product"] = extra_matrix_free_product(pkg, torch, stream, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(P)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "exponent")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    head["ctx"].close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched_problems":
        run_batched(args, rank, world, local_rank)
    elif args.mse:
        run_mse(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
