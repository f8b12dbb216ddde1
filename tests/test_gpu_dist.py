"""The sharded macro iteration on one GPU: two shards of the quadrature points, solved through
fehmm_rve_solve_list and assembled with zeros outside each shard, sum to the full iteration.
(The collectives themselves are covered by the gloo ranks of test_dist_gloo.py.)"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_two_shards_sum_to_the_full_iteration():
    import torch

    import paper_1908_08292_gb300 as fe
    from paper_1908_08292_gb300.dist import Shard, ShardedIteration
    dev = torch.device("cuda:0")
    p = synth.biaxial_shear_2d(macro=4, rve=8, macro_y=8)  # 128 qps, one RVE each
    n_qp, d = p.n_qp, 2
    u = torch.zeros(2 * 5 * 9, dtype=torch.float64, device=dev)
    u[torch.tensor(p.dirichlet_dofs, device=dev)] = torch.tensor(p.dirichlet_end / p.n_steps, device=dev)

    def context():
        ctx = fe.Context(2, "mixed")
        ctx.add_rves(p.rve_n, p.rve_phase, p.rve_E, p.rve_nu)
        ctx.bind_qps(p.qp_rve)
        ctx.macro_create(list(p.macro_n))
        ctx.macro_set_dirichlet(p.dirichlet_dofs, p.dirichlet_end)
        return ctx

    full = context()
    ref = ShardedIteration(full, Shard(0, 1, 0, 32, 4), n_qp, d, dev)
    ref(u, fe.SOLVE_FROM_COMMITTED)
    torch.cuda.synchronize()
    assert int((ref.st == 0).sum()) == n_qp

    ctx = context()
    dofs = np.full(n_qp, 2 * 8 * 8)
    parts = [ShardedIteration(ctx, Shard.make(r, 2, dofs, 4), n_qp, d, dev) for r in range(2)]
    for s in parts:
        s.solve_local(u, fe.SOLVE_FROM_COMMITTED)
        ctx.macro_assemble(s.P, s.A, s.f, s.K)
    torch.cuda.synchronize()
    for s in parts:
        m = torch.tensor(s.shard.local_mask(n_qp), device=dev)
        assert torch.equal(s.P[m], ref.P[m]) and torch.equal(s.A[m], ref.A[m])  # same kernel per point
        assert not s.P[~m].any()  # points of the other shard are never written
    f = parts[0].f + parts[1].f
    K = parts[0].K + parts[1].K
    assert torch.allclose(f, ref.f, rtol=0, atol=1e-13 * float(ref.f.abs().max()))
    assert torch.allclose(K, ref.K, rtol=0, atol=1e-13 * float(ref.K.abs().max()))
    full.close()
    ctx.close()
