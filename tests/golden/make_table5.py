"""Writes tests/golden/table5_*.txt: the reference BLUP of the ill-conditioned
accuracy study (Sec. 8.2, Table 5) for each (alpha, theta) row, computed by
the oracle's extended-precision dense BLUP (oracle.dense_mp, 100 digits; 90
and 150 digits agree to every FP64 digit on the hardest row) on the seeded
unit-disk workload (workloads.unit_disk_gaussian).  Calls only the oracle and
the input generators.  Run from the repository root:

    python tests/golden/make_table5.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import dense_mp  # noqa: E402

DPS = 100


def path_for(alpha, theta):
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), f"table5_a{alpha:g}_t{theta:g}.txt")


def main():
    for alpha, theta in wl.TABLE5_ROWS:
        P = wl.unit_disk_gaussian(alpha, theta)
        y, b, g, res = dense_mp.dense_blup_mp(P.points, P.Z, P.targets, P.w, theta, dps=DPS)
        with open(path_for(alpha, theta), "w") as f:
            f.write(f"# Gaussian-kernel BLUP on the unit disk (Sec. 8.2, Table 5), alpha={alpha:g} theta={theta:g}:\n")
            f.write(f"# workloads.unit_disk_gaussian(alpha, theta), N={P.N}, w={P.w}, no nugget; reference by\n")
            f.write(f"# oracle.dense_mp.dense_blup_mp at {DPS} digits (saddle-point residual {float(res):.1e}).\n")
            f.write("# yhat: predictions at the targets; beta: GLS coefficients in the oracle's monomial order.\n")
            f.write("yhat " + " ".join(repr(float(v)) for v in y) + "\n")
            f.write("beta " + " ".join(repr(float(v)) for v in b) + "\n")
        print("wrote", path_for(alpha, theta), flush=True)


if __name__ == "__main__":
    main()
