"""Micro-benchmark of the PCG operator product C~_W u (Sec. 6, Eq. 17).

Builds the multilevel basis and assembles C~_W for a seeded dense-pattern
problem (all level pairs admissible, tau = infinity), then times
``mlb_cw_matvec_dev`` on the device with CUDA events on the context's stream.
The panels are larger than the L2 cache at the default size, so every call
streams them from HBM.  With ``--matrix-free`` the product is the three-step
W (C (W^T u)) + eta u whose middle step is an N x N kernel sum (the
high-dimensional workload: 262,144 points in [0,1]^10, nu = 5/2, w = 2, leaf
128).  One JSON line per precision:

    python -m paper_1701_00285_gb300.matvec_bench --n 32768 --precision mixed --reps 20
    python -m paper_1701_00285_gb300.matvec_bench --matrix-free --n 262144 --precision mixed --reps 3
"""
from __future__ import annotations

import argparse
import json
import math


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=32768, help="observations")
    ap.add_argument("--precision", default="mixed,fp64", help="comma list of mixed, fp64")
    ap.add_argument("--reps", type=int, default=20, help="timed products")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--leaf-size", type=int, default=None, help="default: the workload's leaf size")
    ap.add_argument("--matrix-free", action="store_true", help="d = 10 three-step product")
    ap.add_argument("--variant", type=int, default=None,
                    help="product form: symmetric storage 0 loads, 1 bulk copies; matrix-free kernel sum 0..5 "
                         "launch shapes, 6 tensor cores; default: the autotuned one")
    a = ap.parse_args(argv)

    import torch
    import workloads as wl
    from .binding import Context

    P = wl.uniform_10d(N=a.n, M=512) if a.matrix_free else wl.heldout_5d(N=a.n, M=512)
    leaf = a.leaf_size or P.leaf_size
    st = torch.cuda.Stream()
    for prec in a.precision.split(","):
        c = Context(prec, leaf_size=leaf, matrix_free=a.matrix_free)
        try:
            c.set_stream(st.cuda_stream)
            c.build_basis(P.points, P.w)
            c.assemble(P.nu, P.rho, P.nugget, math.inf)
            if a.variant is not None and prec == "mixed":
                c.set_product_variant(a.variant)
            nw = c.nwav
            with torch.cuda.stream(st):
                u = torch.randn(nw, dtype=torch.float64, device="cuda",
                                generator=torch.Generator("cuda").manual_seed(1))
                o = torch.empty_like(u)
            st.synchronize()
            for _ in range(a.warmup):
                c.cw_matvec_dev(u.data_ptr(), o.data_ptr())
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(a.reps):
                c.cw_matvec_dev(u.data_ptr(), o.data_ptr())
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / max(a.reps, 1)
            if a.matrix_free:
                # the kernel sum dominates: N^2 point pairs per product
                pairs = a.n * a.n
                print(json.dumps({"precision": prec, "n": a.n, "d": P.points.shape[1], "nwav": nw,
                                  "matrix_free": True, "variant": c.info()["product_variant"], "ms": ms, "pairs": pairs,
                                  "pairs_per_s": pairs / (ms / 1000.0)}), flush=True)
            else:
                vb = 4 if prec == "mixed" else 8
                inf = c.info()
                # tau = infinity makes the pattern dense: nwav^2 entries.  Algorithmic
                # bytes: every entry the product needs once (each symmetric pair once
                # when the storage is symmetric), u read and C~_W u written.
                nnz = inf["nnz_unique"] if inf["symmetric"] else nw * nw
                algo = nnz * vb + 2 * nw * 8
                print(json.dumps({"precision": prec, "n": a.n, "nwav": nw, "nnz": nnz,
                                  "symmetric": inf["symmetric"], "variant": inf["product_variant"],
                                  "stored_values": inf["product_values"],
                                  "ms": ms, "algorithmic_bytes": algo, "GBps": algo / ms / 1e6}), flush=True)
        finally:
            c.close()


if __name__ == "__main__":
    main()
