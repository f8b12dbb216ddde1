"""End-to-end surrogate on the GPU: training data from the library's RVE solves, training with
its BF16 kernels, evaluation with the trust region and the fallback.  A small grid (6^3) of the
fixed two-inclusion microstructure keeps it to seconds.  The test shows what the trained network
gains over the method without it: the surrogate's stresses are an order of magnitude closer to the
RVE solves than the base law's, at a cost far below the RVE solves it replaces."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_surrogate_accuracy_gain_and_speed():
    import torch

    from paper_1908_08292_gb300 import surrogate as su
    torch.cuda.set_device(0)
    one = su.fixed_rve_context(1, grid=6)
    lam0, mu0, Ca = su.base_law(one)
    sp = su.SurrogateParams(lam0, mu0, 0.35, 0.01 * (lam0 + 2 * mu0), 0.3)
    sp.set_Ca(Ca)
    ctx = su.fixed_rve_context(2048, grid=6)
    x, ty, tg, P, W, dropped = su.generate(ctx, sp, synth.stretch_ball(81, 8192, 0.3))
    assert dropped == 0
    Uh = synth.stretch_ball(82, 2048, 0.3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, _, Ph, _, _ = su.generate(ctx, sp, Uh, drop_failed=False)
    torch.cuda.synchronize()
    t_rve = time.perf_counter() - t0
    mlp = su.MLP(4096)
    mlp.set_params(su.init_params(83))
    hist = su.train(mlp, x, ty, tg, epochs=300, batch=2048)
    assert hist[-1] < 0.01 * hist[0]
    sp.set_origin(mlp)
    n = 2048
    F = torch.tensor(Uh.reshape(n, 9), device="cuda")
    Ps = torch.zeros(n, 9, dtype=torch.float64, device="cuda")
    As = torch.zeros(n, 81, dtype=torch.float64, device="cuda")
    ins = torch.zeros(n, dtype=torch.int32, device="cuda")
    work = torch.zeros(su.work_floats(n), dtype=torch.float32, device="cuda")
    su.surrogate_eval(mlp, sp, F, Ps, As, None, ins, work)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    su.surrogate_eval(mlp, sp, F, Ps, As, None, ins, work)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    e = su.stress_errors(Ps.cpu().numpy(), Ph.cpu().numpy(), 1e-3)
    zero = su.MLP(n)
    zero.set_params(np.zeros(su.n_params(), np.float32))
    sp0 = su.SurrogateParams(lam0, mu0, 0.35, 0.01 * (lam0 + 2 * mu0), 0.3)
    sp0.set_Ca(Ca)
    su.surrogate_eval(zero, sp0, F, Ps, As, None, ins, work)
    torch.cuda.synchronize()
    e0 = su.stress_errors(Ps.cpu().numpy(), Ph.cpu().numpy(), 1e-3)
    rms, rms0 = np.sqrt((e ** 2).mean()), np.sqrt((e0 ** 2).mean())
    assert ins.cpu().numpy().all()  # every sample lies in the trust region it was drawn from
    assert rms < 0.1 * rms0, (rms, rms0)
    assert rms < 3e-3, rms
    assert t_sur < 0.05 * t_rve, (t_sur, t_rve)

    # the polynomial part fitted to the same targets already takes most of the base law's error
    spp = su.SurrogateParams(lam0, mu0, 0.35, 0.01 * (lam0 + 2 * mu0), 0.3)
    spp.set_Ca(Ca)
    typ, tgp = ty.clone(), tg.clone()
    su.fit_poly(spp, x, typ, tgp)
    su.surrogate_eval(zero, spp, F, Ps, As, None, ins, work)
    torch.cuda.synchronize()
    rms_p = np.sqrt((su.stress_errors(Ps.cpu().numpy(), Ph.cpu().numpy(), 1e-3) ** 2).mean())
    assert rms_p < rms0 / 3, (rms_p, rms0)
    # and what it leaves is smaller than what the network had to learn without it
    assert float((tgp.double() ** 2).sum()) < float((tg.double() ** 2).sum()) / 9


def test_fallback_replaces_points_outside_trust_region():
    """Points outside the trust region get exactly the full RVE solution; inside, the surrogate."""
    import torch

    from paper_1908_08292_gb300 import select
    from paper_1908_08292_gb300 import surrogate as su
    torch.cuda.set_device(0)
    n = 64
    ctx = su.fixed_rve_context(n, grid=4)
    F = synth.random_F(91, n, 3, 0.3)
    Ft = torch.tensor(F.reshape(n, 9), device="cuda")
    P_full, A_full, _, st = su.rve_solve_batch(ctx, Ft, with_tangent=True, with_energy=False, stages=2)
    sp = su.SurrogateParams(0.7, 0.5, 0.35, 0.01, 0.25)
    mlp = su.MLP(n)
    mlp.set_params(su.init_params(92))
    P = torch.zeros(n, 9, dtype=torch.float64, device="cuda")
    A = torch.zeros(n, 81, dtype=torch.float64, device="cuda")
    ins = torch.zeros(n, dtype=torch.int32, device="cuda")
    work = torch.zeros(su.work_floats(n), dtype=torch.float32, device="cuda")
    su.surrogate_eval(mlp, sp, Ft, P, A, None, ins, work)
    P_sur = P.clone()
    lst = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    select(ins, 0, lst, cnt)
    st2 = torch.zeros(n, dtype=torch.int32, device="cuda")
    it2 = torch.zeros(n, 4, dtype=torch.int32, device="cuda")
    from paper_1908_08292_gb300 import SOLVE_FROM_COMMITTED
    ctx.rve_solve_list(Ft, P, A, st2, it2, SOLVE_FROM_COMMITTED, lst, cnt)
    torch.cuda.synchronize()
    inside = ins.cpu().numpy().astype(bool)
    k = int(cnt.item())
    assert k == (~inside).sum() and 0 < k < n
    assert np.array_equal(np.sort(lst[:k].cpu().numpy()), np.nonzero(~inside)[0])
    np.testing.assert_array_equal(P.cpu().numpy()[inside], P_sur.cpu().numpy()[inside])
    out = ~inside & (st.cpu().numpy() == 0)
    np.testing.assert_allclose(P.cpu().numpy()[out], P_full.cpu().numpy()[out], rtol=0, atol=1e-7)
