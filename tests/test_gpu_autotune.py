"""The solver-settings autotuner (fehmm_autotune): it times candidate settings on a sample of the
bound points, keeps the fastest that converges, caches the choice by problem class and device,
and the batch solved with the chosen settings still matches the FP64 oracle (mixed precision,
1e-5 on P and A)."""
import numpy as np
import pytest

import synth
from gpu_harness import rel_err
from oracle.rve import PeriodicRVE

pytestmark = pytest.mark.gpu


def _solve(ctx, F, n_qp, d):
    import torch
    dev = torch.device("cuda:0")
    P = torch.zeros(n_qp, d * d, dtype=torch.float64, device=dev)
    A = torch.zeros(n_qp, d ** 4, dtype=torch.float64, device=dev)
    st = torch.full((n_qp,), -1, dtype=torch.int32, device=dev)
    it = torch.zeros(n_qp, 4, dtype=torch.int32, device=dev)
    ctx.rve_solve(F, P, A, st, it)
    torch.cuda.synchronize()
    return P.cpu().numpy(), A.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("dim", [2, 3])
def test_autotune_then_oracle_parity_and_cache(dim, tmp_path):
    import torch

    import paper_1908_08292_gb300 as fe
    if dim == 2:
        p = synth.biaxial_shear_2d(macro=4, rve=32)  # 64 points of 32x32 RVEs
    else:
        p = synth.uniaxial_3d_uneven(macro=1, sizes=(8, 12), n_rve=8)  # 8 points, uneven 8^3 / 12^3
    d, n_qp = p.dim, p.n_qp
    Fs = synth.random_F(801 + dim, n_qp, d, 0.08)
    F = torch.tensor(Fs.reshape(n_qp, d * d), dtype=torch.float64, device="cuda")
    cache = str(tmp_path / "tune.txt")
    with fe.Context(d, "mixed") as ctx:
        ctx.add_rves(p.rve_n, p.rve_phase, p.rve_E, p.rve_nu)
        ctx.bind_qps(p.qp_rve)
        r = ctx.autotune(F, n_sample=min(n_qp, 16), cache_path=cache)
        assert r["from_cache"] == 0 and r["candidates"] >= 5 and r["seconds_per_solve"] > 0
        o = ctx.options
        assert (o.precond, o.mg_reuse) == (r["precond"], r["mg_reuse"])
        assert o.mg_omega == pytest.approx(r["mg_omega"]) and o.cg_rtol == pytest.approx(r["cg_rtol"])
        # the current fluctuations are as before the trials (all zero here)
        assert float(ctx.fluctuations().abs().max().item()) == 0.0
        P, A, st, it = _solve(ctx, F, n_qp, d)
    assert (st == 0).all()
    for q in (0, n_qp // 2, n_qp - 1):
        r_ = p.qp_rve[q]
        ref = PeriodicRVE(int(p.rve_n[r_]), d, p.rve_phase[r_], p.rve_E[r_], p.rve_nu[r_]).solve(
            Fs[q], rtol=1e-13, atol=1e-16)
        assert rel_err(P[q], ref["P"], 1e-3) < 1e-5 and rel_err(A[q], ref["A"], 1e-3) < 1e-5
    # a second context of the same problem class takes the cached choice without timing
    with fe.Context(d, "mixed") as ctx2:
        ctx2.add_rves(p.rve_n, p.rve_phase, p.rve_E, p.rve_nu)
        ctx2.bind_qps(p.qp_rve)
        r2 = ctx2.autotune(F, cache_path=cache)
        assert r2["from_cache"] == 1 and r2["candidates"] == 0
        assert (r2["precond"], r2["mg_reuse"]) == (r["precond"], r["mg_reuse"])
        assert r2["mg_omega"] == r["mg_omega"] and r2["cg_rtol"] == r["cg_rtol"]
