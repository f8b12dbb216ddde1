"""Load-step drivers for the two-level Newton schemes (oracle; test infrastructure only).

Algorithm 1 / Sec. 5.1 (nested): every macro iteration runs each RVE Newton to
convergence.  Algorithm 2 / Sec. 5.2 (alternating): every macro iteration runs
exactly one micro Newton iteration per RVE.  In both schemes the fluctuation of
the last micro state is superimposed on the updated macro field as the start
value (Sec. 5.1 warm start, Sec. 5.2), and the RVE pass that follows the final
macro update is the "accuracy polish" of Sec. 5.1/5.2: the loop below always
ends with an RVE pass at the final macro displacement, and the alternating
scheme adds one more micro iteration after the macro residual has converged.
The algorithms print "while residual < tolerance"; read as "while residual >
tolerance".  The first macro iterate of a load step is the previous converged
displacement with the Dirichlet dofs set to their new values, or (predictor=True; the
paper is silent on the start of a load step) the tangent predictor: with the tangent K
of the last converged state, the Dirichlet increment d and the interior correction
delta solving K_ff delta = -(K d)_f of the linearised macro problem, u + d + delta.
"""
from __future__ import annotations

import numpy as np

from .macro import MacroMesh
from .rve import PeriodicRVE


def build_rves(problem):
    return [PeriodicRVE(int(problem.rve_n[r]), problem.dim, problem.rve_phase[r],
                        problem.rve_E[r], problem.rve_nu[r]) for r in range(len(problem.rve_phase))]


def rve_batch(rves, qp_rve, Fbar, w, rtol=1e-10, atol=1e-14, max_iter=30, max_steps=None, tangent=True):
    """One RVE solve per macro qp; returns Pbar, Abar, Wbar, new fluctuations, status, iters."""
    n_qp, d = Fbar.shape[0], Fbar.shape[1]
    P = np.zeros((n_qp, d, d))
    A = np.zeros((n_qp, d, d, d, d))
    W = np.zeros(n_qp)
    status = np.zeros(n_qp, dtype=np.int32)
    iters = np.zeros(n_qp, dtype=np.int32)
    w_new = []
    for q in range(n_qp):
        out = rves[qp_rve[q]].solve(Fbar[q], w[q], rtol, atol, max_iter, max_steps, tangent)
        w_new.append(out["w"])
        status[q] = out["status"]
        iters[q] = out["newton_iters"]
        if "P" in out:
            P[q], W[q] = out["P"], out["W"]
            if tangent:
                A[q] = out["A"]
    return P, A, W, w_new, status, iters


def run(problem, scheme="nested", n_steps=None, macro_rtol=1e-10, macro_atol=1e-13, max_macro=40,
        micro_rtol=None, micro_atol=1e-14, steps_to_run=None, log=None, predictor=False):
    """Run the FE-HMM load steps.  Returns per-step records (u, Pbar, Abar, iteration counts)."""
    mesh = MacroMesh(problem.macro_n)
    rves = build_rves(problem)
    d = problem.dim
    n_steps = problem.n_steps if n_steps is None else n_steps
    micro_rtol = problem.newton_tol if micro_rtol is None else micro_rtol
    u = np.zeros(mesh.n_dof)
    w_comm = [np.zeros(rves[problem.qp_rve[q]].n_dof) for q in range(problem.n_qp)]
    records = []
    last = n_steps if steps_to_run is None else steps_to_run
    max_steps = 1 if scheme == "alternating" else None
    K = None
    for k in range(1, last + 1):
        lam = k / n_steps
        if predictor:
            if K is None:  # tangent at the start state
                _, A0, _, _, _, _ = rve_batch(rves, problem.qp_rve, mesh.qp_F(u), w_comm, micro_rtol, micro_atol)
                _, K = mesh.assemble(np.zeros((problem.n_qp, d, d)), A0)
            dvec = np.zeros(mesh.n_dof)
            dvec[problem.dirichlet_dofs] = problem.dirichlet_end / n_steps
            delta, _ = mesh.solve_increment(K, K @ dvec, problem.dirichlet_dofs)
            u += dvec + delta
        u[problem.dirichlet_dofs] = lam * problem.dirichlet_end
        w = [x.copy() for x in w_comm]
        hist, micro_iters = [], []
        f0 = None
        converged = False
        for it in range(max_macro + 1):
            Fbar = mesh.qp_F(u)
            P, A, W, w, status, iters = rve_batch(rves, problem.qp_rve, Fbar, w, micro_rtol, micro_atol,
                                                  max_steps=max_steps)
            micro_iters.append(int(iters.sum()))
            if np.any(status > 1):
                raise RuntimeError(f"RVE failure at step {k}, macro iteration {it}: {np.unique(status)}")
            f, K = mesh.assemble(P, A)
            free = np.setdiff1d(np.arange(mesh.n_dof), problem.dirichlet_dofs)
            fn = float(np.linalg.norm(f[free]))
            f0 = fn if f0 is None else f0
            hist.append(fn)
            if log:
                log(f"step {k} macro {it} |f|={fn:.3e} micro_iters={int(iters.sum())}")
            if fn <= max(macro_rtol * f0, macro_atol):
                converged = True
                break
            du, _ = mesh.solve_increment(K, f, problem.dirichlet_dofs)
            u += du
        if scheme == "alternating":  # final micro iteration after macro convergence (Sec. 5.2)
            Fbar = mesh.qp_F(u)
            P, A, W, w, status, iters = rve_batch(rves, problem.qp_rve, Fbar, w, micro_rtol, micro_atol,
                                                  max_steps=1)
            micro_iters.append(int(iters.sum()))
            _, K = mesh.assemble(P, A)  # the tangent of the final state (the next step's predictor)
        w_comm = w
        records.append({"step": k, "u": u.copy(), "P": P, "A": A, "W": W, "macro_iters": len(hist) - 1,
                        "macro_hist": hist, "micro_iters": micro_iters, "converged": converged})
    return records, mesh
