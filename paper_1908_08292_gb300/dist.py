"""Data-parallel sharding of the macro quadrature points over ranks (one process per GPU).

The RVE problems of different macro quadrature points are independent (Sec. 3.2: one micro
problem per point), so a rank owns a contiguous block of macro elements together with their
quadrature points (qp = element * points_per_element + local index) and their fluctuation state,
and solves only those RVEs.  Macro assembly (Eq. f_I^int, Eq. Assem_k_T_IK_mac) is linear in
Pbar and Abar: each rank assembles with its own points' Pbar, Abar and zeros elsewhere, and one
sum over ranks of the residual f and of the CSR tangent values K gives the global system — the
single exchange of a macro iteration.  Rank 0 solves the (small) macro system and broadcasts the
correction, so every rank holds the same macro state by construction.

The surrogate network trains data-parallel the same way: every rank takes its slice of each
global batch (batch_slice), its loss carries the weight 1/(global batch), so one sum of the
gradient buffer over the ranks (allreduce_gradient, about 200 KB in FP32) gives every rank the
full-batch gradient and identical AdamW steps.

Host logic only (partition, qp lists, the collectives on tensors); every arithmetic step of an
iteration runs in the library's kernels.  The collectives work on CUDA tensors with NCCL and on
CPU tensors with gloo.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def partition_elements(cost: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Split elements 0..n-1 into `world` contiguous ranges [e0, e1) of nearly equal total cost
    (cost[e] >= 0, e.g. the summed RVE dofs of the element's points).  Boundaries are the
    elements at which the running cost first reaches k/world of the total; every range is
    non-empty when n >= world."""
    cost = np.asarray(cost, dtype=np.float64)
    n = cost.size
    if world < 1 or n < world:
        raise ValueError(f"cannot split {n} elements over {world} ranks")
    csum = np.cumsum(cost)
    total = csum[-1] if n else 0.0
    bounds = [0]
    for k in range(1, world):
        b = int(np.searchsorted(csum, total * k / world, side="left")) + 1 if total > 0 else (n * k) // world
        b = min(max(b, bounds[-1] + 1), n - (world - k))  # keep every range non-empty
        bounds.append(b)
    bounds.append(n)
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


def element_cost(rve_dofs_per_qp: np.ndarray, nq: int) -> np.ndarray:
    """Per-element cost = sum of the RVE dofs of its nq points (qp = element * nq + l)."""
    return np.asarray(rve_dofs_per_qp, dtype=np.float64).reshape(-1, nq).sum(axis=1)


def batch_slice(s0: int, batch: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [a, b) of the global batch [s0, s0 + batch) that `rank` of `world` trains on
    (contiguous, sizes differing by at most one)."""
    a = s0 + (batch * rank) // world
    b = s0 + (batch * (rank + 1)) // world
    return a, b


def allreduce_gradient(grad, world: int):
    """Sum a gradient tensor over the ranks, in place (no-op on one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(grad, op=dist.ReduceOp.SUM)


def qp_range_list(e0: int, e1: int, nq: int) -> np.ndarray:
    return np.arange(e0 * nq, e1 * nq, dtype=np.int32)


@dataclass
class Shard:
    """One rank's share of the macro quadrature points."""
    rank: int
    world: int
    e0: int
    e1: int
    nq: int

    @classmethod
    def make(cls, rank, world, rve_dofs_per_qp, nq):
        ranges = partition_elements(element_cost(rve_dofs_per_qp, nq), world)
        e0, e1 = ranges[rank]
        return cls(rank, world, e0, e1, nq)

    @property
    def qps(self) -> np.ndarray:
        return qp_range_list(self.e0, self.e1, self.nq)

    @property
    def n_local(self) -> int:
        return (self.e1 - self.e0) * self.nq

    def local_mask(self, n_qp: int) -> np.ndarray:
        m = np.zeros(n_qp, dtype=bool)
        m[self.e0 * self.nq:self.e1 * self.nq] = True
        return m

    def reduce_system(self, f, K):
        """Sum the partial macro residual and tangent values over ranks (in place)."""
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(f, op=dist.ReduceOp.SUM)
            dist.all_reduce(K, op=dist.ReduceOp.SUM)

    def share_correction(self, du):
        """Make rank 0's macro correction every rank's (in place)."""
        if self.world > 1:
            import torch.distributed as dist
            dist.broadcast(du, src=0)


class ShardedIteration:
    """One macro iteration of the nested scheme on this rank's share of the points:
    Fbar at all points (cheap), RVE solves of the local points only (fehmm_rve_solve_list),
    partial assembly, the sum over ranks, the macro solve on rank 0 and its broadcast."""

    def __init__(self, ctx, shard: Shard, n_qp: int, dim: int, device):
        import torch
        self.ctx, self.shard = ctx, shard
        d = dim
        self.F = torch.zeros(n_qp, d * d, dtype=torch.float64, device=device)
        self.P = torch.zeros(n_qp, d * d, dtype=torch.float64, device=device)  # zero outside the shard
        self.A = torch.zeros(n_qp, d ** 4, dtype=torch.float64, device=device)
        self.st = torch.zeros(n_qp, dtype=torch.int32, device=device)
        self.it = torch.zeros(n_qp, 4, dtype=torch.int32, device=device)
        self.lst = torch.tensor(shard.qps, dtype=torch.int32, device=device)
        self.cnt = torch.tensor([shard.n_local], dtype=torch.int32, device=device)
        _, _, n_rows, nnz = ctx.macro_csr()
        self.f = torch.zeros(n_rows, dtype=torch.float64, device=device)
        self.K = torch.zeros(nnz, dtype=torch.float64, device=device)
        self.du = torch.zeros(n_rows, dtype=torch.float64, device=device)
        self.info = torch.zeros(3, dtype=torch.float64, device=device)

    def solve_local(self, u, flags):
        self.ctx.macro_qp_F(u, self.F)
        self.ctx.rve_solve_list(self.F, self.P, self.A, self.st, self.it, flags, self.lst, self.cnt)

    def assemble_and_solve(self, rtol=1e-10):
        self.ctx.macro_assemble(self.P, self.A, self.f, self.K)
        self.shard.reduce_system(self.f, self.K)
        if self.shard.rank == 0:
            self.ctx.macro_solve(self.K, self.f, self.du, self.info, rtol=rtol)
        self.shard.share_correction(self.du)

    def __call__(self, u, flags, rtol=1e-10):
        self.solve_local(u, flags)
        self.assemble_and_solve(rtol)
