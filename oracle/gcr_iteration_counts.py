"""Iteration counts of the oracle's unpreconditioned GCR on the benchmark's
field distribution, for the CPU baseline of bench.py.

Test infrastructure only (see ``oracle/__init__``).

The benchmark solves point sources on 32^3x64 and 24^3x48 (U = exp(0.15 i H),
c_sw 1.9, kappa 0.1300) to 1e-3 and, for the bias correction, to 1e-10
starting from the 1e-3 solution (Sec. 2.1, eqs. caa1/caa2).  A complete
unpreconditioned oracle solve at those sizes does not finish in reasonable
time on host cores, so this script completes the same solves on a smaller
field drawn from the same distribution (same eps, c_sw, kappa; its own seed)
and records the iteration counts; bench.py multiplies them by the time per
oracle GCR iteration measured on that field and scaled by volume.  (The count
of an unpreconditioned solver grows with the volume as the lowest modes move
down, so counts taken on the smaller lattice understate the full-size cost:
the CPU figure is favourable to the CPU.)  The committed file was written
with --dims 16 8 8 8.  On larger copies the unpreconditioned restarted GCR
stagnates: with --dims 24 12 12 12 it stopped at its 20,000-iteration cap
with relative residuals of 3.7e-3 (aiming at 1e-3) and then 1.6e-3 (aiming
at 1e-10), after 4.9 hours on the build machine's cores; so the counts of the
smaller field understate the oracle's cost at the benchmark's sizes by a
large factor.

    python -m oracle.gcr_iteration_counts        # writes oracle/gcr_iteration_counts.json
    python -m oracle.gcr_iteration_counts --dims 24 12 12 12 --out <path>   # a smaller copy
"""
from __future__ import annotations

import json
import os
import time

from paper_1605_00564_gb300 import synth

from .dirac import Operator
from .solve import gcr

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "gcr_iteration_counts.json")

CASE = dict(dims=(32, 16, 16, 16), eps=0.15, csw=1.9, kappa=0.1300, seed=160500568, bc_t=-1,
            src=(0, 0, 0, 0), spin=0, colour=0, nkv=24, sloppy_tol=1e-3, exact_tol=1e-10)


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=None, help="T X Y Z (default: 32 16 16 16)")
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    c = dict(CASE)
    if args.dims:
        c["dims"] = tuple(args.dims)
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    op = Operator(U, c["kappa"], c["csw"], c["bc_t"])
    eta = synth.point_source(c["dims"], c["src"], c["spin"], c["colour"])
    t0 = time.perf_counter()
    psi, n_s, r_s = gcr(op, eta, tol=c["sloppy_tol"], nkv=c["nkv"])
    t1 = time.perf_counter()
    _, n_e, r_e = gcr(op, eta, tol=c["exact_tol"], nkv=c["nkv"], psi0=psi)
    t2 = time.perf_counter()
    rec = dict(c)
    rec.update(dict(iters_sloppy=int(n_s), residual_sloppy=float(r_s), iters_exact_from_sloppy=int(n_e),
                    residual_exact=float(r_e), seconds_sloppy=round(t1 - t0, 1), seconds_exact=round(t2 - t1, 1),
                    solver="oracle.solve.gcr (restarted GCR, nkv 24, FP64, unpreconditioned)"))
    with open(args.out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
