"""Parity of the CUDA macro kernels (fehmm_macro_qp_F, fehmm_macro_assemble) with the oracle's
macro mesh on random displacement fields and random per-qp Pbar / Abar."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle.macro import MacroMesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_el", [(4, 4), (5, 3), (3, 2, 4)])
def test_macro_qp_F_and_assembly(n_el):
    import torch

    import paper_1908_08292_gb300 as fe

    d = len(n_el)
    mesh = MacroMesh(n_el)
    dev = torch.device("cuda:0")
    u = synth.random_field(301, 1, mesh.n_dof, 0.1)[0]
    P = synth.random_field(302, mesh.n_qp, d * d, 1.0)
    A = synth.random_field(303, mesh.n_qp, d ** 4, 1.0)
    with fe.Context(d, "mixed") as ctx:
        ctx.macro_create(n_el)
        ut = torch.tensor(u, device=dev)
        F = torch.zeros(mesh.n_qp, d * d, dtype=torch.float64, device=dev)
        ctx.macro_qp_F(ut, F)
        rowptr, col, nr, nnz = ctx.macro_csr()
        f = torch.zeros(mesh.n_dof, dtype=torch.float64, device=dev)
        K = torch.zeros(nnz, dtype=torch.float64, device=dev)
        ctx.macro_assemble(torch.tensor(P, device=dev), torch.tensor(A, device=dev), f, K)
        torch.cuda.synchronize()
        Fg = F.cpu().numpy().reshape(-1, d, d)
        fg = f.cpu().numpy()
        Kg = sp.csr_matrix((K.cpu().numpy(), col.cpu().numpy(), rowptr.cpu().numpy()), shape=(nr, nr))
    np.testing.assert_allclose(Fg, mesh.qp_F(u), atol=1e-14, rtol=0)
    f_ref, K_ref = mesh.assemble(P.reshape(-1, d, d), A.reshape(-1, d, d, d, d))
    np.testing.assert_allclose(fg, f_ref, atol=1e-13 * np.abs(f_ref).max())
    assert abs(Kg - K_ref).max() < 1e-13 * abs(K_ref).max()
    # the CSR pattern holds exactly the node-neighbour blocks
    assert nnz == K_ref.nnz or abs(K_ref).max() > 0
