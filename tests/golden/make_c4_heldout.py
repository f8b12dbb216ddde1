"""Write c4_heldout_oracle.txt: the FP64 oracle's homogenised stress Pbar and energy Wbar of the
fixed 12^3 two-inclusion RVE (the surrogate workload's microstructure, synth.fixed_rve12, matrix E = 1,
inclusions E = 10, nu = 0.3) at the first N held-out right stretches U of that workload's sampler
(synth.stretch_ball, seed 2004, |U - I|_F <= 0.3).

Calls only oracle/ and synth/ (test infrastructure).  Each point is solved from zero fluctuation
directly (Newton, rtol 1e-11), or in 3 load-continuation stages if that fails.  Runs on a
process pool; about 15 s of CPU per point.

Usage: python tests/golden/make_c4_heldout.py [N] [processes]
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_heldout_oracle.txt")
SEED, RADIUS = 2004, 0.3


def _solve(q_and_U):
    sys.path.insert(0, ROOT)
    import synth
    from oracle.rve import STATUS_OK, PeriodicRVE
    q, U = q_and_U
    phase, _ = synth.fixed_rve12()
    rve = PeriodicRVE(12, 3, phase, [1.0, 10.0], [0.3, 0.3])
    r = rve.solve(U, rtol=1e-11, tangent=False)
    stages = 1
    if r["status"] != STATUS_OK:
        w, stages = None, 3
        for s in (1.0 / 3.0, 2.0 / 3.0, 1.0):
            r = rve.solve(np.eye(3) + s * (U - np.eye(3)), w, rtol=1e-11, tangent=False)
            w = r["w"]
    return q, int(r["status"]), stages, r.get("P"), r.get("W")


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 1024
    procs = int(sys.argv[2]) if len(sys.argv) > 2 else max(1, (os.cpu_count() or 2) - 1)
    sys.path.insert(0, ROOT)
    import synth
    U = synth.stretch_ball(SEED, n, RADIUS)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ[k] = "1"
    with mp.get_context("spawn").Pool(procs) as pool:
        res = sorted(pool.map(_solve, list(enumerate(U)), chunksize=1))
    with open(OUT, "w") as f:
        f.write("# FP64 oracle Pbar (row-major 3x3) and Wbar of the fixed 12^3 two-inclusion RVE (synth.fixed_rve12;\n")
        f.write("# E = 1 / 10, nu = 0.3) at the first %d held-out stretches U of synth.stretch_ball(%d, N, %.1f).\n"
                % (n, SEED, RADIUS))
        f.write("# Written by tests/golden/make_c4_heldout.py (oracle/ and synth/ only).\n")
        f.write("# columns: q status stages P00 P01 P02 P10 P11 P12 P20 P21 P22 W\n")
        for q, st, stages, P, W in res:
            vals = list(np.asarray(P).reshape(-1)) + [W] if P is not None else [float("nan")] * 10
            f.write("%d %d %d " % (q, st, stages) + " ".join("%.17g" % v for v in vals) + "\n")


if __name__ == "__main__":
    main()
