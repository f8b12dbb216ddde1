"""Multi-rank sharding of the macro quadrature points, on CPU ranks (gloo, world size 2).

The partition and the collectives of paper_1908_08292_gb300.dist are exercised with the FP64
oracle standing in for the kernels of each rank (RVE solves of the local points, assembly with
zeros outside the shard): the summed partial systems and the broadcast correction must equal the
single-process macro iteration."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1908_08292_gb300.dist import Shard, element_cost, partition_elements


def test_partition_covers_every_element_once_and_balances():
    for seed, n, world in [(1, 37, 1), (2, 64, 2), (3, 100, 3), (4, 9, 4), (5, 128, 8), (6, 5, 5)]:
        cost = 1.0 + 9.0 * synth.uniform(seed, np.arange(n), 1)[:, 0]
        r = partition_elements(cost, world)
        assert r[0][0] == 0 and r[-1][1] == n and len(r) == world
        assert all(a < b for a, b in r) and all(r[k][1] == r[k + 1][0] for k in range(world - 1))
        per = [cost[a:b].sum() for a, b in r]
        assert max(per) <= cost.sum() / world + cost.max() + 1e-12, (seed, per)
    with pytest.raises(ValueError):
        partition_elements(np.ones(3), 4)


def test_uneven_rve_sizes_shift_the_boundary():
    """Elements whose points carry 16^3 RVEs weigh 8x those with 8^3: the cut follows the dofs."""
    nq = 8
    dofs = np.repeat([3 * 8 ** 3] * 6 + [3 * 16 ** 3] * 2, nq)
    ranges = partition_elements(element_cost(dofs, nq), 2)
    assert ranges == [(0, 7), (7, 8)]
    s = Shard.make(1, 2, dofs, nq)
    assert list(s.qps) == list(range(56, 64)) and s.local_mask(64).sum() == 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    return synth.biaxial_shear_2d(macro=2, rve=8, seed=1002)


def _iteration_inputs():
    from oracle.macro import MacroMesh
    p = _problem()
    mesh = MacroMesh(p.macro_n)
    u = np.zeros(mesh.n_dof)
    u[p.dirichlet_dofs] = p.dirichlet_end / p.n_steps  # first iterate of load step 1
    return p, mesh, u


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from oracle.driver import build_rves, rve_batch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, mesh, u = _iteration_inputs()
        dofs = np.array([p.dim * int(p.rve_n[r]) ** p.dim for r in p.qp_rve])
        shard = Shard.make(rank, world, dofs, mesh.nq)
        F = mesh.qp_F(u)
        P = np.zeros((p.n_qp, 2, 2))
        A = np.zeros((p.n_qp, 2, 2, 2, 2))
        loc = shard.qps
        rves = build_rves(p)
        Pl, Al, _, _, st, _ = rve_batch(rves, p.qp_rve[loc], F[loc], [None] * loc.size, rtol=1e-13)
        assert (st == 0).all()
        P[loc], A[loc] = Pl, Al
        f, K = mesh.assemble(P, A)
        ft = torch.tensor(f)
        Kt = torch.tensor(K.toarray().reshape(-1))
        shard.reduce_system(ft, Kt)
        du = torch.zeros(mesh.n_dof, dtype=torch.float64)
        if rank == 0:
            import scipy.sparse as sp
            d, _ = mesh.solve_increment(sp.csr_matrix(Kt.numpy().reshape(mesh.n_dof, mesh.n_dof)), ft.numpy(),
                                        p.dirichlet_dofs)
            du.copy_(torch.tensor(d))
        shard.share_correction(du)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), f=ft.numpy(), K=Kt.numpy(), du=du.numpy(),
                 e0=shard.e0, e1=shard.e1)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_iteration(tmp_path):
    import torch.multiprocessing as mp

    from oracle.driver import build_rves, rve_batch
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    p, mesh, u = _iteration_inputs()
    F = mesh.qp_F(u)
    P, A, _, _, st, _ = rve_batch(build_rves(p), p.qp_rve, F, [None] * p.n_qp, rtol=1e-13)
    f, K = mesh.assemble(P, A)
    du, _ = mesh.solve_increment(K, f, p.dirichlet_dofs)
    r = [np.load(os.path.join(tmp_path, f"rank{k}.npz")) for k in range(world)]
    assert int(r[0]["e1"]) == int(r[1]["e0"]) and int(r[0]["e0"]) == 0 and int(r[1]["e1"]) == mesh.n_el
    for k in range(world):
        np.testing.assert_allclose(r[k]["f"], f, rtol=0, atol=1e-13)
        np.testing.assert_allclose(r[k]["K"], K.toarray().reshape(-1), rtol=0, atol=1e-12)
        np.testing.assert_allclose(r[k]["du"], du, rtol=1e-11, atol=1e-14)
    assert np.array_equal(r[0]["du"], r[1]["du"])  # the broadcast makes the macro state identical


def _grad_rank_main(rank, world, port, out_dir):
    """One data-parallel training step's gradient: this rank's slice of the global batch, the
    oracle's double-backward gradient standing in for the library's kernels, loss weights
    1/(global batch), then the sum over ranks."""
    import torch
    import torch.distributed as dist

    from oracle import mlp as omlp
    from paper_1908_08292_gb300.dist import allreduce_gradient, batch_slice
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        params, x, ty, tg, B = _grad_inputs()
        a, b = batch_slice(0, B, rank, world)
        G = omlp.param_grad(params, x[a:b], ty[a:b], tg[a:b], 1.0 / B, 0.5 / B)
        flat = torch.tensor(np.concatenate([np.asarray(G[k]).reshape(-1) for k in sorted(G)]))
        allreduce_gradient(flat, world)
        np.save(os.path.join(out_dir, f"grad{rank}.npy"), flat.numpy())
    finally:
        dist.destroy_process_group()


def _grad_inputs():
    from oracle import mlp as omlp
    params = omlp.init_params(91)
    B = 37  # odd: the two slices differ in size
    x = synth.random_field(92, B, 6, 0.8)
    ty = synth.random_field(93, 1, B, 1.0)[0]
    tg = synth.random_field(94, B, 6, 1.0)
    return params, x, ty, tg, B


def test_two_gloo_ranks_sum_to_the_full_batch_gradient(tmp_path):
    """Data-parallel surrogate training: the per-rank gradients of the rank slices, summed by
    allreduce_gradient, equal the full-batch gradient on every rank."""
    import torch.multiprocessing as mp

    from oracle import mlp as omlp
    from paper_1908_08292_gb300.dist import batch_slice
    world, port = 2, _free_port()
    mp.spawn(_grad_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    params, x, ty, tg, B = _grad_inputs()
    G = omlp.param_grad(params, x, ty, tg, 1.0 / B, 0.5 / B)
    full = np.concatenate([np.asarray(G[k]).reshape(-1) for k in sorted(G)])
    got = [np.load(os.path.join(tmp_path, f"grad{k}.npy")) for k in range(world)]
    assert [batch_slice(0, B, r, world) for r in range(world)] == [(0, 18), (18, 37)]
    for g in got:
        np.testing.assert_allclose(g, full, rtol=1e-12, atol=1e-14 * np.abs(full).max())
    assert np.array_equal(got[0], got[1])
