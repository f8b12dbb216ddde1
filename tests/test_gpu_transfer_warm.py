"""Warm-started tangent transfer (fehmm_options.transfer_warm): each point's transfer solutions
are kept as load-step state and start the next solve's transfer PCG.  The result must still
match the FP64 oracle at the same tolerances, need fewer transfer iterations on a nearby
deformation, and commit/rollback must restore that state exactly (a repeated solve after a
rollback repeats the same iteration counts and results bit for bit)."""
import numpy as np
import pytest

import synth
from gpu_harness import rel_err
from oracle.rve import PeriodicRVE

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
STRICT = {2: dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-8, cond_rtol=1e-11),
          3: dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-9, cond_rtol=1e-11)}


def _ctx(dim, precision, sizes, phases, E, nu, qp_rve, warm):
    import paper_1908_08292_gb300 as fe
    opts = dict(STRICT[dim]) if precision == "fp64" else {}
    ctx = fe.Context(dim, precision, transfer_warm=int(warm), **opts)
    ctx.add_rves(sizes, phases, E, nu)
    ctx.bind_qps(np.asarray(qp_rve, dtype=np.int32))
    return ctx


def _solve(ctx, Fs, flags=0):
    import torch
    n, d = Fs.shape[0], Fs.shape[1]
    dev = torch.device("cuda:0")
    F = torch.tensor(Fs.reshape(n, d * d), dtype=torch.float64, device=dev)
    P = torch.zeros(n, d * d, dtype=torch.float64, device=dev)
    A = torch.zeros(n, d ** 4, dtype=torch.float64, device=dev)
    st = torch.full((n,), -1, dtype=torch.int32, device=dev)
    it = torch.zeros(n, 4, dtype=torch.int32, device=dev)
    ctx.rve_solve(F, P, A, st, it, flags=flags)
    torch.cuda.synchronize()
    return P.cpu().numpy(), A.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (2, "mixed"), (3, "fp64"), (3, "mixed")])
def test_warm_transfer_matches_oracle_with_fewer_iterations(dim, precision):
    if dim == 2:
        sizes = [8, 16, 32]
        u = synth.uniform(901, np.arange(3), 4)
        phases = [synth.phase_from_inclusions(n, 2, [u[k, :2]], [0.15 + 0.2 * u[k, 2]]) for k, n in enumerate(sizes)]
        E = [[1.0, 5.0 + 40.0 * u[k, 3]] for k in range(3)]
    else:
        sizes = [4, 8, 12]
        u = synth.uniform(902, np.arange(3), 4)
        phases = [synth.phase_from_inclusions(n, 3, [u[k, :3]], [0.2 + 0.1 * u[k, 3]]) for k, n in enumerate(sizes)]
        E = [[1.0, 10.0]] * 3
    nu = [[0.3, 0.3]] * 3
    qp_rve = [0, 1, 2]
    F1 = synth.random_F(903 + dim, 3, dim, 0.08)
    F2 = F1 + 0.01 * (synth.random_F(905 + dim, 3, dim, 1.0) - np.eye(dim))  # the next macro iterate, say
    out = {}
    for warm in (0, 1):
        ctx = _ctx(dim, precision, sizes, phases, E, nu, qp_rve, warm)
        try:
            _solve(ctx, F1)
            out[warm] = _solve(ctx, F2)
        finally:
            ctx.close()
    refs = [PeriodicRVE(sizes[r], dim, phases[r], E[r], nu[r]).solve(F2[q], rtol=1e-14, atol=1e-16)
            for q, r in enumerate(qp_rve)]
    for warm in (0, 1):
        P, A, st, it = out[warm]
        for q, ref in enumerate(refs):
            assert st[q] == 0
            assert rel_err(P[q], ref["P"], 1e-3) < TOL[precision]
            assert rel_err(A[q], ref["A"], 1e-3) < TOL[precision], (warm, q, rel_err(A[q], ref["A"], 1e-3))
    # a strong (multigrid) preconditioner converges fast from any start, so a start value saves a
    # few iterations per solve: most at the mixed tolerance (1e-6), least at the strict FP64 one
    cold_it, warm_it = out[0][3][:, 2].sum(), out[1][3][:, 2].sum()
    assert warm_it < (0.8 if precision == "mixed" else 0.95) * cold_it, (warm_it, cold_it)


def test_rollback_restores_the_kept_transfer_state():
    sizes = [16]
    phase = synth.phase_from_inclusions(16, 2, [[0.4, 0.6]], [0.3])
    ctx = _ctx(2, "mixed", sizes, [phase], [[1.0, 20.0]], [[0.3, 0.3]], [0, 0], 1)
    try:
        F0 = synth.random_F(911, 2, 2, 0.05)
        _solve(ctx, F0)
        ctx.commit()
        F1 = F0 + 0.02 * (synth.random_F(912, 2, 2, 1.0) - np.eye(2))
        a = _solve(ctx, F1, flags=2)
        x_after = ctx.transfer_state().clone()
        ctx.rollback()
        b = _solve(ctx, F1, flags=2)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
        assert bool((ctx.transfer_state() == x_after).all())
    finally:
        ctx.close()
