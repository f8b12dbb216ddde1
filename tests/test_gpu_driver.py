"""GPU load-step driver (Algorithms 1 and 2) and macro solve against the FP64 oracle."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import driver as odriver
from oracle import material as mat
from oracle.macro import MacroMesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_el", [(6, 5), (52, 48)])
def test_macro_solve_matches_direct_solve(n_el):
    """(6, 5): 84 rows, 3 blocks; (52, 48): 5194 rows, every SM a block and several rows per
    lane group."""
    import torch

    import paper_1908_08292_gb300 as fe

    mesh = MacroMesh(n_el)
    lam, mu = mat.lame(3.0, 0.3)
    F = synth.random_F(501, mesh.n_qp, 2, 0.05)
    P, A = mat.P_of_F(F, lam, mu), mat.A_of_F(F, lam, mu)
    f_ref, K_ref = mesh.assemble(P, A)
    fixed = np.nonzero(np.isclose(mesh.X[:, 0], 0.0))[0]
    dofs = np.concatenate([2 * fixed, 2 * fixed + 1]).astype(np.int32)
    dev = torch.device("cuda:0")
    with fe.Context(2, "fp64") as ctx:
        ctx.macro_create(n_el)
        ctx.macro_set_dirichlet(dofs, np.zeros(dofs.size))
        rowptr, col, nr, nnz = ctx.macro_csr()
        Pt, At = torch.tensor(P.reshape(-1, 4), device=dev), torch.tensor(A.reshape(-1, 16), device=dev)
        f = torch.zeros(nr, dtype=torch.float64, device=dev)
        K = torch.zeros(nnz, dtype=torch.float64, device=dev)
        du = torch.zeros(nr, dtype=torch.float64, device=dev)
        info = torch.zeros(3, dtype=torch.float64, device=dev)
        ctx.macro_assemble(Pt, At, f, K)
        ctx.macro_solve(K, f, du, info, rtol=1e-13, max_it=20000)
        torch.cuda.synchronize()
        du, info = du.cpu().numpy(), info.cpu().numpy()
    free = np.setdiff1d(np.arange(mesh.n_dof), dofs)
    ref = np.zeros(mesh.n_dof)
    ref[free] = spla.spsolve(K_ref[free][:, free].tocsc(), -f_ref[free])
    assert info[2] == 0
    assert abs(info[0] - np.linalg.norm(f_ref[free])) < 1e-12 * np.linalg.norm(f_ref)
    # CG error <= condition number x relative residual: about 1e4 x 1e-13 on the larger mesh
    np.testing.assert_allclose(du, ref, atol=(1e-9 if mesh.n_dof < 1000 else 1e-8) * np.abs(ref).max())
    assert np.all(du[dofs] == 0)


def test_macro_solve_repeatable_with_one_block_per_sm():
    """The cooperative macro CG with the largest grid (one block per SM) run many times on the same
    system: every run must give a bit-identical correction and the same iteration count.  Each
    block adds the grid's partial sums itself, so a block that read another call's partials (the
    reuse of one partial buffer by back-to-back grid reductions) would take different step
    lengths from the others; the reductions alternate between two buffers to exclude that."""
    import torch

    import paper_1908_08292_gb300 as fe

    n_el = (52, 48)  # 5194 rows: more rows than 32 x (number of SMs), so one block per SM
    mesh = MacroMesh(n_el)
    lam, mu = mat.lame(3.0, 0.3)
    F = synth.random_F(502, mesh.n_qp, 2, 0.05)
    P, A = mat.P_of_F(F, lam, mu), mat.A_of_F(F, lam, mu)
    fixed = np.nonzero(np.isclose(mesh.X[:, 0], 0.0))[0]
    dofs = np.concatenate([2 * fixed, 2 * fixed + 1]).astype(np.int32)
    dev = torch.device("cuda:0")
    assert torch.cuda.get_device_properties(dev).multi_processor_count * 32 < mesh.n_dof
    with fe.Context(2, "fp64") as ctx:
        ctx.macro_create(n_el)
        ctx.macro_set_dirichlet(dofs, np.zeros(dofs.size))
        _, _, nr, nnz = ctx.macro_csr()
        f = torch.zeros(nr, dtype=torch.float64, device=dev)
        K = torch.zeros(nnz, dtype=torch.float64, device=dev)
        ctx.macro_assemble(torch.tensor(P.reshape(-1, 4), device=dev), torch.tensor(A.reshape(-1, 16), device=dev),
                           f, K)
        runs = 40
        du = torch.zeros(runs, nr, dtype=torch.float64, device=dev)
        info = torch.zeros(runs, 3, dtype=torch.float64, device=dev)
        for k in range(runs):
            ctx.macro_solve(K, f, du[k], info[k], rtol=1e-12, max_it=20000)
        torch.cuda.synchronize()
        du, info = du.cpu().numpy(), info.cpu().numpy()
    assert np.all(info[:, 2] == 0)
    assert np.all(info[:, 1] == info[0, 1]) and info[0, 1] > 10
    assert np.array_equal(du, np.broadcast_to(du[0], du.shape))


@pytest.mark.parametrize("scheme", ["nested", "alternating"])
def test_uniaxial_2d_load_steps_match_oracle(scheme):
    """All ten load steps of the 4x4 Q1 uniaxial problem (stretch to 10 %) against the oracle's Algorithm 1
    or 2."""
    from paper_1908_08292_gb300.driver import LoadStepDriver

    p = synth.uniaxial_2d_small()
    steps = 10
    ref, mesh = odriver.run(p, scheme=scheme, steps_to_run=steps, micro_rtol=1e-12)
    drv = LoadStepDriver(p, precision="fp64", scheme=scheme, newton_rtol=1e-12, newton_atol=1e-15, cg_rtol=1e-9,
                         cond_rtol=1e-11)
    try:
        for k in range(1, steps + 1):
            rec = drv.load_step(k)
            assert rec["converged"]
            u = drv.u.cpu().numpy()
            P = drv.P.cpu().numpy().reshape(-1, 2, 2)
            r = ref[k - 1]
            assert np.abs(u - r["u"]).max() < 1e-9 * np.abs(r["u"]).max()
            assert np.abs(P - r["P"]).max() < 1e-9 * np.abs(r["P"]).max()
            assert abs(rec["macro_iters"] - r["macro_iters"]) <= (0 if scheme == "nested" else 1)
    finally:
        drv.close()


def test_uniaxial_2d_tangent_predictor_matches_oracle():
    """Load steps that start from the tangent predictor (the Dirichlet increment's load on the
    last converged tangent and the interior correction it implies) against the oracle's driver
    with the same predictor: same macro iterations, same displacements and stresses."""
    from paper_1908_08292_gb300.driver import LoadStepDriver

    p = synth.uniaxial_2d_small()
    steps = 4
    ref, mesh = odriver.run(p, scheme="nested", steps_to_run=steps, micro_rtol=1e-12, predictor=True)
    drv = LoadStepDriver(p, precision="fp64", scheme="nested", newton_rtol=1e-12, newton_atol=1e-15, cg_rtol=1e-9,
                         cond_rtol=1e-11, predictor=True)
    try:
        for k in range(1, steps + 1):
            rec = drv.load_step(k)
            assert rec["converged"]
            u = drv.u.cpu().numpy()
            P = drv.P.cpu().numpy().reshape(-1, 2, 2)
            r = ref[k - 1]
            assert np.abs(u - r["u"]).max() < 1e-9 * np.abs(r["u"]).max()
            assert np.abs(P - r["P"]).max() < 1e-9 * np.abs(r["P"]).max()
            assert rec["macro_iters"] == r["macro_iters"]
    finally:
        drv.close()


def test_graph_replay_equals_eager():
    from paper_1908_08292_gb300.driver import LoadStepDriver

    p = synth.uniaxial_2d_small()
    out = []
    for graphs in (False, True):
        drv = LoadStepDriver(p, precision="mixed", graphs=graphs)
        try:
            recs = [drv.load_step(k) for k in (1, 2)]
            out.append((drv.u.cpu().numpy(), [r["macro_iters"] for r in recs]))
        finally:
            drv.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
