"""Two-level Newton load-step driver on the GPU: Algorithm 1 (nested) and Algorithm 2
(alternating) of the paper, Sec. 5.

Host control flow only: every step of a macro iteration is a library kernel launched through
the C ABI — Dirichlet data and u += du (fehmm_macro_apply_dirichlet / fehmm_macro_update),
Fbar at the quadrature points, the batched RVE solves, the macro assembly and the macro CG
solve.  The host reads back three numbers per macro iteration (|f_free|, CG iterations, CG
status) to decide convergence.

Iteration structure of one load step (Sec. 5.1 / 5.2):
  u[Dirichlet] <- t * u_hat, du <- 0
  repeat:  u += du;  Fbar(u);  RVE solves (nested: to convergence; alternating: one micro
           Newton iteration) starting from the last micro state (the committed one on the
           first iteration: the warm start of Sec. 5.1);  assemble f, K;  solve K du = -f
  until |f_free| <= max(rtol |f_free at the first iteration|, atol)
The RVE pass of the last iteration is the "accuracy polish" of Sec. 5.1; the alternating
scheme adds one more micro iteration at the converged u (Sec. 5.2).  Then commit.

With graphs=True one macro iteration is captured into two CUDA graphs (first iteration of a
step, later iterations) and replayed.
"""
from __future__ import annotations

import time

import numpy as np

from . import SOLVE_FROM_COMMITTED, Context, FehmmError


class LoadStepDriver:
    def __init__(self, problem, precision=None, scheme="nested", graphs=False, macro_rtol=1e-10, macro_atol=1e-13,
                 max_macro=40, solve_rtol=1e-12, shard=None, predictor=False, **options):
        import torch

        if scheme not in ("nested", "alternating"):
            raise FehmmError(f"unknown scheme {scheme}")
        self.p = problem
        self.scheme = scheme
        self.macro_rtol, self.macro_atol, self.max_macro = macro_rtol, macro_atol, max_macro
        self.solve_rtol = solve_rtol
        precision = precision or problem.precision
        opts = dict(newton_rtol=problem.newton_tol)
        opts.update(options)
        if scheme == "alternating":
            opts["max_newton"] = 1
        d = problem.dim
        self.ctx = Context(d, precision, **opts)
        self.ctx.add_rves(problem.rve_n, problem.rve_phase, problem.rve_E, problem.rve_nu)
        self.ctx.bind_qps(problem.qp_rve)
        self.ctx.macro_create(list(problem.macro_n))
        self.ctx.macro_set_dirichlet(problem.dirichlet_dofs, problem.dirichlet_end)
        _, _, n_rows, nnz = self.ctx.macro_csr()
        dev = torch.device("cuda", torch.cuda.current_device())
        n_qp = problem.n_qp
        f64, i32 = torch.float64, torch.int32
        self.u = torch.zeros(n_rows, dtype=f64, device=dev)
        self.du = torch.zeros(n_rows, dtype=f64, device=dev)
        self.F = torch.zeros(n_qp, d * d, dtype=f64, device=dev)
        self.P = torch.zeros(n_qp, d * d, dtype=f64, device=dev)
        self.A = torch.zeros(n_qp, d ** 4, dtype=f64, device=dev)
        self.st = torch.zeros(n_qp, dtype=i32, device=dev)
        self.it = torch.zeros(n_qp, 4, dtype=i32, device=dev)
        self.f = torch.zeros(n_rows, dtype=f64, device=dev)
        self.K = torch.zeros(nnz, dtype=f64, device=dev)
        self.info = torch.zeros(3, dtype=f64, device=dev)
        # tangent predictor of a load step (predictor=True): the Dirichlet increment's load on the
        # last converged tangent, g = K d, and the correction K_ff delta = -g_f
        self.predictor = predictor
        self.g = torch.zeros(n_rows, dtype=f64, device=dev)
        self.K_valid = False
        # data-parallel ranks (dist.Shard): this rank solves only its points' RVEs, the partial
        # macro systems are summed over ranks, rank 0 solves and broadcasts du and the CG info
        self.shard = shard
        if shard is not None:
            self.lst = torch.tensor(shard.qps, dtype=i32, device=dev)
            self.cnt = torch.tensor([shard.n_local], dtype=i32, device=dev)
        self.scale = 0.0
        self.graphs = graphs
        self._g = {}
        self._warm = set()
        # optional instrumentation: when a list, every batched RVE solve is bracketed by a pair of
        # CUDA timing events on the current stream, appended here (eager runs only)
        self.rve_events = None
        # optional instrumentation: when a list, the per-point iteration counts of every batched
        # RVE solve are copied here (for operation counts; not used by the iteration itself)
        self.iter_log = None

    # ------------------------------------------------------------ one iteration
    def _constitutive(self, first):
        """Pbar, Abar at every macro point: one batched RVE solve (overridden by the surrogate path)."""
        flags = SOLVE_FROM_COMMITTED if first else 0
        if self.shard is None:
            self.ctx.rve_solve(self.F, self.P, self.A, self.st, self.it, flags=flags)
        else:
            self.ctx.rve_solve_list(self.F, self.P, self.A, self.st, self.it, flags, self.lst, self.cnt)

    def _iteration(self, first, solve=True):
        import torch
        c = self.ctx
        c.macro_update(self.u, self.du)
        c.macro_qp_F(self.u, self.F)
        if self.rve_events is not None:
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record()
            self._constitutive(first)
            ev[1].record()
            self.rve_events.append(ev)
        else:
            self._constitutive(first)
        if self.iter_log is not None:
            self.iter_log.append(self.it.clone())
        c.macro_assemble(self.P, self.A, self.f, self.K)
        if self.shard is not None:
            self.shard.reduce_system(self.f, self.K)
        if solve:
            self._solve(self.f)

    def _run(self, first):
        import torch
        if not self.graphs or self.rve_events is not None or self.iter_log is not None:
            self._iteration(first)
            return
        key = bool(first)
        if key not in self._warm:  # run each variant once eagerly (module loading, attributes)
            self._warm.add(key)
            self._iteration(first)
            return
        if key not in self._g:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._iteration(first)
            self._g[key] = g
        self._g[key].replay()

    def _solve(self, f):
        """du = -K_ff^-1 f_f on rank 0, shared with every rank (with the CG info)."""
        if self.shard is None or self.shard.rank == 0:
            self.ctx.macro_solve(self.K, f, self.du, self.info, rtol=self.solve_rtol)
        if self.shard is not None:
            self.shard.share_correction(self.du)
            self.shard.share_correction(self.info)

    def _predict(self, new_scale):
        """Tangent predictor: with the tangent K of the last converged state (one RVE pass at the
        current state first if there is none yet), the Dirichlet increment d = (new_scale - scale)
        u_hat and the interior correction delta with K_ff delta = -(K d)_f; the first macro
        iteration then starts from u + d + delta instead of concentrating d in the boundary
        elements.  Returns the number of RVE passes it ran (0 or 1)."""
        c = self.ctx
        passes = 0
        if not self.K_valid:
            c.macro_qp_F(self.u, self.F)
            self._constitutive(True)
            c.macro_assemble(self.P, self.A, self.f, self.K)
            if self.shard is not None:
                self.shard.reduce_system(self.f, self.K)
            passes = 1
        c.macro_dirichlet_load(self.K, new_scale - self.scale, self.g)
        self._solve(self.g)
        c.macro_apply_dirichlet(self.u, None, new_scale)  # u[D] = new values; du keeps delta
        return passes

    def state(self):
        """Copy of the load-step state (macro u, committed fluctuations and kept transfer solutions, last
        tangent) to repeat a step."""
        xs = self.ctx.transfer_state(committed=True)
        return (self.u.clone(), self.ctx.fluctuations(committed=True).clone(), None if xs is None else xs.clone(),
                self.K.clone(), self.K_valid, self.scale)

    def restore(self, st):
        u, w, xs, K, kv, scale = st
        self.u.copy_(u)
        self.ctx.fluctuations(committed=True).copy_(w)
        if xs is not None:
            self.ctx.transfer_state(committed=True).copy_(xs)
        self.ctx.rollback()
        self.K.copy_(K)
        self.K_valid, self.scale = kv, scale

    # --------------------------------------------------------------- load step
    def load_step(self, k, commit=True):
        """Run load step k (load factor k / n_steps); returns a record of the iterations.  With
        commit=False the converged fluctuations stay current only (the committed state of the
        previous step is kept, so the step can be repeated after restoring u and a rollback)."""
        import torch
        t0 = time.perf_counter()
        new_scale = k / self.p.n_steps
        extra = 0
        if self.predictor:
            extra = self._predict(new_scale)
        else:
            self.ctx.macro_apply_dirichlet(self.u, self.du, new_scale)
        self.scale = new_scale
        hist, cg_its, micro = [], [], []
        f0 = None
        converged = False
        for it in range(self.max_macro + 1):
            self._run(first=(it == 0))
            info = self.info.cpu().numpy()
            status = self.st.cpu().numpy()
            if np.any(status > 1):
                raise FehmmError(f"RVE failure at step {k}, macro iteration {it}: statuses {np.unique(status)}")
            micro.append(int(self.it[:, 0].sum().item()))
            fn = float(info[0])
            f0 = fn if f0 is None else f0
            hist.append(fn)
            cg_its.append(int(info[1]))
            if fn <= max(self.macro_rtol * f0, self.macro_atol):
                converged = True
                break
        # the last iteration's du is not applied: the state stays at the converged u
        self.ctx.macro_apply_dirichlet(self.u, self.du, self.scale)
        if self.scheme == "alternating":  # final micro iteration at the converged u (Sec. 5.2)
            self._iteration(first=False, solve=False)
            micro.append(int(self.it[:, 0].sum().item()))
        self.K_valid = True  # the last pass assembled the tangent at the converged state
        if commit:
            self.ctx.commit()
        torch.cuda.synchronize()
        return {"step": k, "macro_iters": len(hist) - 1, "macro_hist": hist, "macro_cg": cg_its,
                "micro_newton": micro, "rve_passes": len(micro) + extra, "converged": converged,
                "seconds": time.perf_counter() - t0}

    def run(self, steps=None):
        steps = self.p.n_steps if steps is None else steps
        return [self.load_step(k) for k in range(1, steps + 1)]

    def close(self):
        self.ctx.close()
