"""GPU test of the no-allocation entry point fehmm_rve2d_solve_fp64_noalloc.

That entry point serves callers that cannot call cudaMalloc (allocator-free runtimes that hand
the library only pre-registered buffers, code running while a memory pool is torn down or
resized, deployments that need a footprint fixed at load time): it keeps its kernel scratch in a
static device array instead of allocating.  This test calls it twice in a row through the C ABI
(the second call sees the array and work counter as the first call left them) and checks each
call's stress, tangent and fluctuations against the context-based fehmm_rve_solve in FP64 mode,
at the FP64 parity tolerance of the other GPU tests (1e-10 relative).  This file is collected
last so that a run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_harness import gpu_batch, rel_err

pytestmark = pytest.mark.gpu

STRICT = dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-8, cond_rtol=1e-11)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_context_entry_point_on_two_calls():
    import torch

    import paper_1908_08292_gb300 as fe

    L = fe.lib()
    dev = torch.device("cuda:0")
    n, n_qp = 8, 6
    E, nu = np.array([1.0, 10.0]), np.array([0.3, 0.3])
    phase = synth.phase_from_inclusions(n, 2, [[0.5, 0.5]], [0.25])
    table = np.zeros((4, 2))  # (lambda, mu) per phase, as the paper's material table derives them
    table[:2, 0] = E * nu / ((1 + nu) * (1 - 2 * nu))
    table[:2, 1] = E / (2 * (1 + nu))
    opt = fe.Options()
    assert L.fehmm_default_options(ctypes.byref(opt), 2, fe.PREC_FP64) == 0
    for k, v in STRICT.items():
        setattr(opt, k, v)
    phase_d = torch.tensor(phase, dtype=torch.uint8, device=dev)
    table_d = torch.tensor(table.reshape(-1), dtype=torch.float64, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (401, 402):
        Fs = synth.random_F(seed, n_qp, 2, 0.1)
        ref = gpu_batch(2, "fp64", [n], [phase], [E], [nu], np.zeros(n_qp), Fs, **STRICT)
        F = torch.tensor(Fs.reshape(n_qp, 4), dtype=torch.float64, device=dev)
        w = torch.zeros(n_qp * n * n * 2, dtype=torch.float64, device=dev)
        P = torch.zeros(n_qp, 4, dtype=torch.float64, device=dev)
        A = torch.zeros(n_qp, 16, dtype=torch.float64, device=dev)
        st = torch.full((n_qp,), -1, dtype=torch.int32, device=dev)
        it = torch.zeros(n_qp, 4, dtype=torch.int32, device=dev)
        rc = L.fehmm_rve2d_solve_fp64_noalloc(n_qp, n, 0, _ptr(phase_d), _ptr(table_d), _ptr(w), _ptr(F), _ptr(P),
                                               _ptr(A), _ptr(st), _ptr(it), ctypes.byref(opt), stream)
        assert rc == 0, fe.status_str(rc)
        torch.cuda.synchronize()
        P, A, st = P.cpu().numpy(), A.cpu().numpy(), st.cpu().numpy()
        w = w.cpu().numpy().reshape(n_qp, -1)
        for q in range(n_qp):
            assert st[q] == 0 and ref["status"][q] == 0
            assert rel_err(P[q], ref["P"][q], 1e-3) < 1e-10
            assert rel_err(A[q], ref["A"][q], 1e-3) < 1e-10
            assert np.abs(w[q] - ref["w"][q]).max() < 1e-10
    # a device phase map with an id outside the 4-entry material table: that point is reported
    # with FEHMM_RVE_BAD_PHASE (7) before any table read and left unsolved; the others solve
    bad = np.stack([phase, phase])
    bad[1, 5] = 6
    bad_d = torch.tensor(bad, dtype=torch.uint8, device=dev)
    table2 = torch.tensor(np.stack([table, table]).reshape(-1), dtype=torch.float64, device=dev)
    Fs = synth.random_F(403, 2, 2, 0.05)
    F = torch.tensor(Fs.reshape(2, 4), dtype=torch.float64, device=dev)
    w = torch.zeros(2 * n * n * 2, dtype=torch.float64, device=dev)
    P = torch.full((2, 4), 7.0, dtype=torch.float64, device=dev)
    st = torch.full((2,), -1, dtype=torch.int32, device=dev)
    rc = L.fehmm_rve2d_solve_fp64_noalloc(2, n, 1, _ptr(bad_d), _ptr(table2), _ptr(w), _ptr(F), _ptr(P), None,
                                           _ptr(st), None, ctypes.byref(opt), stream)
    assert rc == 0
    torch.cuda.synchronize()
    st, P = st.cpu().numpy(), P.cpu().numpy()
    assert st[0] == 0 and st[1] == 7 and np.all(P[1] == 7.0)
    # a grid beyond the static scratch is rejected before any launch
    rc = L.fehmm_rve2d_solve_fp64_noalloc(1, 18, 0, _ptr(phase_d), _ptr(table_d), _ptr(table_d), _ptr(table_d),
                                           _ptr(table_d), None, _ptr(table_d), None, ctypes.byref(opt), stream)
    assert rc == -6 and "static scratch" in fe.status_str(rc)
