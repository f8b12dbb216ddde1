"""The surrogate workload's RVE at full size on the GPU against stored FP64 oracle values: the fixed
12^3 two-inclusion RVE (matrix E = 1, inclusions E = 10, nu = 0.3) at the first held-out right
stretches U (|U - I|_F <= 0.3) of the workload's sampler, solved in the library's mixed precision
with the 3-stage load continuation the training-data generator uses.  The homogenised stress is
set by the FP64 residual the Newton loop drives to its tolerance, so it matches the oracle far
below the mixed-mode tangent tolerance; the energy likewise.  Expected values:
tests/golden/c4_heldout_oracle.txt, written by tests/golden/make_c4_heldout.py from oracle/ only."""
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c4_heldout_oracle.txt")


def _golden(n):
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[int(f[0])] = (np.array([float(v) for v in f[3:12]]), float(f[12]))
    return [rows[q] for q in range(n)]


def test_fixed_rve12_matches_stored_oracle_values():
    import torch

    from paper_1908_08292_gb300 import surrogate as su
    n = 64
    ref = _golden(n)
    U = synth.stretch_ball(2004, n, 0.3)
    ctx = su.fixed_rve_context(n)
    F = torch.tensor(U.reshape(n, 9), device="cuda")
    P, _, W, st = su.rve_solve_batch(ctx, F, stages=3)
    P, W, st = P.cpu().numpy(), W.cpu().numpy(), st.cpu().numpy()
    assert np.all(st <= 1), st
    for q in range(n):
        Pr, Wr = ref[q]
        eP = np.linalg.norm(P[q] - Pr) / np.linalg.norm(Pr)
        eW = abs(W[q] - Wr) / abs(Wr)
        assert eP < 1e-9 and eW < 1e-9, (q, eP, eW)
    ctx.close()
