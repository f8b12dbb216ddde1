"""Helpers shared by the GPU tests: run batches through the C-ABI binding and compare with
the FP64 oracle.  Not collected by pytest (no test_ prefix)."""
from __future__ import annotations

import numpy as np


def rel_err(a, b, floor):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor))


def gpu_batch(dim, precision, grid_n, phases, E, nu, qp_rve, Fs, flags=0, w0=None, **opts):
    """One fehmm_rve_solve over the given quadrature points; returns numpy outputs."""
    import torch

    import paper_1908_08292_gb300 as fe

    dev = torch.device("cuda:0")
    n_qp = len(qp_rve)
    d = dim
    with fe.Context(dim, precision, **opts) as ctx:
        ctx.add_rves(grid_n, phases, E, nu)
        ctx.bind_qps(np.asarray(qp_rve, dtype=np.int32))
        if w0 is not None:
            for q in range(n_qp):
                ctx.fluctuation(q).copy_(torch.as_tensor(w0[q], dtype=torch.float64, device=dev))
        F = torch.tensor(np.asarray(Fs).reshape(n_qp, d * d), dtype=torch.float64, device=dev)
        P = torch.zeros(n_qp, d * d, dtype=torch.float64, device=dev)
        A = torch.zeros(n_qp, d ** 4, dtype=torch.float64, device=dev)
        W = torch.zeros(n_qp, dtype=torch.float64, device=dev)
        st = torch.full((n_qp,), -1, dtype=torch.int32, device=dev)
        it = torch.zeros(n_qp, 4, dtype=torch.int32, device=dev)
        ctx.rve_solve(F, P, A, st, it, W, flags=flags)
        torch.cuda.synchronize()
        w = [ctx.fluctuation(q).cpu().numpy().copy() for q in range(n_qp)]
        return {"P": P.cpu().numpy().reshape(n_qp, d, d), "A": A.cpu().numpy().reshape(n_qp, d, d, d, d),
                "W": W.cpu().numpy(), "status": st.cpu().numpy(), "iters": it.cpu().numpy(), "w": w}
