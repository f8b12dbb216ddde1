"""Benchmark of the batched periodic-RVE hot path on one (or N) GB300.

Workload (one "step"): the 2D plane-strain FE-HMM workload with a 32x32 Q1 macro mesh
(4096 macro quadrature points) and one 32x32 Q1 periodic RVE per point (random circular
inclusion, stiffness ratio 5-50), mixed FP32/FP64 precision.  A step is one macro iteration
of the hot path: Fbar at the quadrature points from the macro displacement, the batched RVE
Newton solves with homogenised stress and tangent (starting from the committed fluctuations
of the previous load step), the macro residual/tangent assembly and the macro Newton
correction (GPU CG on the assembled tangent).

Value: RVE solves per second (whole job, all ranks).  Also reported: micro-DOF x Newton
iterations per second.  `--impl reference` times the FP64 CPU oracle on a bounded sample
of the same workload instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--step-index S]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RVE solves/s (micro-DOF*Newton-iter/s reported alongside)"
_SIZE = {"macro": 32, "workload": "c2"}
UNIT = "RVE solves/s"
MACRO, RVE_N, N_STEPS = 32, 32, 20
MACRO_C3, N_STEPS_C3 = 8, 10

# Algorithmic operation counts per unit of the 2D mixed kernel (derivation in the design doc,
# counted from the kernel source, an FMA counting 2).
FP64_FLOP_PER_ELEMENT_RESIDUAL = 290.0   # F, J, F^-T, P and nodal forces at 4 Gauss points + gather
FP32_FLOP_PER_ELEMENT_TANGENT = 1350.0   # 8x8 element tangent at 4 Gauss points + stencil gather
FP32_FLOP_PER_NODE_PCG_ITER = 100.0      # 9-block 2x2 stencil apply + vector updates + 2 dots
FP32_FLOP_PER_ELEMENT_TRANSFER = 1500.0  # energy form of the tangent transfer (4 unit gradients)
FP64_FLOP_PER_ELEMENT_RESIDUAL_3D = 2640.0   # Hex8: 8 Gauss points x (grad, F^-T, P, nodal forces)
FP32_FLOP_PER_ELEMENT_TANGENT_3D = 4200.0    # Gauss-point data + 3x3 diagonal blocks
FP32_FLOP_PER_ELEMENT_APPLY_3D = 4000.0      # matrix-free apply: grad, dP = A:dF, nodal scatter
FP32_FLOP_PER_NODE_PCG_ITER_3D = 30.0        # preconditioner + vector updates + dots
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
FP64_PEAK_TFLOPS = 1.25                              # GB300 nominal FP64


def workload_config(step_index):
    MACRO = _SIZE["macro"]
    if _SIZE["workload"] == "c3":
        return {"workload": f"3D FE-HMM macro {MACRO}^3 Hex8 ({MACRO ** 3 * 8} qps), one periodic Hex8 RVE per qp "
                            f"of 8^3/12^3/16^3 elements (uniform draw), 1-4 spheres (volume fraction 0.1-0.3, "
                            f"stiffness ratio 10), neo-Hookean, mixed FP32/FP64, uneven batch in one persistent "
                            f"launch, macro iteration 1 of load step {step_index}/{N_STEPS_C3} (uniaxial to 20%)",
                "n_qp": MACRO ** 3 * 8, "rve_grid": "8/12/16 mixed", "load_step": step_index,
                "l2": "flushed (256 MB write) between timed steps"}
    return {"workload": f"2D plane-strain FE-HMM macro {MACRO}x{MACRO} Q1 ({MACRO * MACRO * 4} qps), "
                        f"one {RVE_N}x{RVE_N} Q1 periodic RVE per qp (random circular inclusion r~U(0.15,0.35), "
                        f"E ratio log-U[5,50]), neo-Hookean, mixed FP32/FP64, macro iteration 1 of load step "
                        f"{step_index}/{N_STEPS} (biaxial 30% + shear 0.3)",
            "n_qp": MACRO * MACRO * 4, "rve_grid": RVE_N, "micro_dofs_per_rve": 2 * RVE_N * RVE_N,
            "load_step": step_index, "l2": "flushed (256 MB write) between timed steps"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].isdigit():
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def build_problem(step_index):
    """The workload and the macro deformation gradient of the affine first iterate of the step."""
    import synth
    if _SIZE["workload"] == "c3":
        p = synth.config3(macro=_SIZE["macro"])
        F = np.diag([1.0 + 0.2 * step_index / N_STEPS_C3, 1.0, 1.0])
        return p, F
    p = synth.config2(macro=_SIZE["macro"], rve=RVE_N)
    lam = step_index / N_STEPS
    F = np.eye(2) + lam * (p.extra["F_end"] - np.eye(2))
    return p, F


def macro_affine_u(F):
    """u = (F - I) X at the macro nodes (x fastest)."""
    MACRO = _SIZE["macro"]
    d = F.shape[0]
    ax = np.arange(MACRO + 1) / MACRO
    X = np.stack(np.meshgrid(*([ax] * d), indexing="ij"), -1)
    X = X.transpose(*range(d - 1, -1, -1), d).reshape(-1, d)
    return (X @ (F - np.eye(d)).T).reshape(-1)


def flops_3d(p, iters):
    """FP64 and FP32 algorithmic flops of one 3D batch solve from the per-qp iteration counts."""
    el = np.array([int(p.rve_n[r]) ** 3 for r in p.qp_rve], dtype=np.float64)
    newton = iters[:, 0].astype(np.float64)
    cg = iters[:, 1].astype(np.float64) + iters[:, 2].astype(np.float64)
    f64 = ((newton + 1) * FP64_FLOP_PER_ELEMENT_RESIDUAL_3D * el).sum()
    f32 = ((newton + 1) * FP32_FLOP_PER_ELEMENT_TANGENT_3D * el
           + (cg + 9) * (FP32_FLOP_PER_ELEMENT_APPLY_3D + FP32_FLOP_PER_NODE_PCG_ITER_3D) * el).sum()
    return f64, f32


def flops_2d(n, iters):
    """FP64 and FP32 algorithmic flops of one RVE batch solve from the per-qp iteration counts."""
    el = n * n
    newton = iters[:, 0].astype(np.float64)
    cg = iters[:, 1].astype(np.float64) + iters[:, 2].astype(np.float64)
    f64 = ((newton + 1) * FP64_FLOP_PER_ELEMENT_RESIDUAL * el).sum()
    f32 = ((newton + 1) * FP32_FLOP_PER_ELEMENT_TANGENT * el + cg * FP32_FLOP_PER_NODE_PCG_ITER * el
           + FP32_FLOP_PER_ELEMENT_TRANSFER * el).sum()
    return f64, f32


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1908_08292_gb300 as fe

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    fe.lib()
    p, Fload = build_problem(args.step_index)
    n_qp = p.n_qp
    opts = {k: v for k, v in (("cg_rtol", args.cg_rtol), ("cond_rtol", args.cond_rtol)) if v is not None}
    d = p.dim
    ctx = fe.Context(d, "mixed", **opts)
    ctx.add_rves(p.rve_n, p.rve_phase, p.rve_E, p.rve_nu)
    ctx.bind_qps(p.qp_rve)
    ctx.macro_create([_SIZE["macro"]] * d)
    ctx.macro_set_dirichlet(p.dirichlet_dofs, p.dirichlet_end)
    _, _, n_rows, nnz = ctx.macro_csr()
    u_h = torch.tensor(macro_affine_u(Fload), dtype=torch.float64).pin_memory()
    u = u_h.to(dev)
    F = torch.empty(n_qp, d * d, dtype=torch.float64, device=dev)
    P = torch.empty(n_qp, d * d, dtype=torch.float64, device=dev)
    A = torch.empty(n_qp, d ** 4, dtype=torch.float64, device=dev)
    st = torch.empty(n_qp, dtype=torch.int32, device=dev)
    it = torch.empty(n_qp, 4, dtype=torch.int32, device=dev)
    f = torch.empty(n_rows, dtype=torch.float64, device=dev)
    K = torch.empty(nnz, dtype=torch.float64, device=dev)
    du = torch.empty(n_rows, dtype=torch.float64, device=dev)
    info = torch.empty(3, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ctx.macro_qp_F(u, F)
        ctx.rve_solve(F, P, A, st, it, flags=fe.SOLVE_FROM_COMMITTED)
        ctx.macro_assemble(P, A, f, K)
        ctx.macro_solve(K, f, du, info, rtol=1e-10)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launches
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(5)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            e0, e1, e2, e3, e4 = ev[k]
            e0.record(stream)
            ctx.macro_qp_F(u, F)
            e1.record(stream)
            ctx.rve_solve(F, P, A, st, it, flags=fe.SOLVE_FROM_COMMITTED)
            e2.record(stream)
            ctx.macro_assemble(P, A, f, K)
            e3.record(stream)
            ctx.macro_solve(K, f, du, info, rtol=1e-10)
            e4.record(stream)
        torch.cuda.synchronize()
    launches = ctx.launches - launches0
    step_ms = [ev[k][0].elapsed_time(ev[k][4]) for k in range(args.steps)]
    rve_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    t_step = sum(step_ms) / 1e3
    if world > 1:
        tt = torch.tensor([t_step], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
        dist.barrier()
    status = st.cpu().numpy()
    iters = it.cpu().numpy()
    ok = int((status == 0).sum())
    # ---- end-to-end through the public API with host buffers (H2D of u, D2H of results)
    f_h = torch.empty(n_rows, dtype=torch.float64).pin_memory()
    K_h = torch.empty(nnz, dtype=torch.float64).pin_memory()
    P_h = torch.empty(n_qp, d * d, dtype=torch.float64).pin_memory()
    A_h = torch.empty(n_qp, d ** 4, dtype=torch.float64).pin_memory()
    s_h = torch.empty(n_qp, dtype=torch.int32).pin_memory()
    e2e_ms = []
    for k in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u.copy_(u_h, non_blocking=True)
        step()
        f_h.copy_(du, non_blocking=True)
        K_h.copy_(K, non_blocking=True)
        P_h.copy_(P, non_blocking=True)
        A_h.copy_(A, non_blocking=True)
        s_h.copy_(st, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = u_h.numel() * 8
    d2h = (n_rows + nnz + n_qp * (d * d + d ** 4)) * 8 + n_qp * 4
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    n_total = n_qp * world
    value = n_total / (t_step / args.steps)
    dofs = np.array([d * int(p.rve_n[r]) ** d for r in p.qp_rve], dtype=np.float64)
    dof_iter = float((dofs * iters[:, 0].astype(np.float64)).sum()) * world / (t_step / args.steps)
    f64, f32 = flops_2d(RVE_N, iters) if d == 2 else flops_3d(p, iters)
    t_rve = statistics.mean(rve_ms) / 1e3
    ach_eq = (f32 + f64 * FP32_PEAK_TFLOPS / FP64_PEAK_TFLOPS) / t_rve / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed: FP64 residual/sums, FP32 tangent/PCG)",
        "data": "synthetic (seeded generator, config-2 shapes)", "config": workload_config(args.step_index),
        "micro_dof_newton_iter_per_s": dof_iter,
        "rve_status_ok": ok, "newton_iters_mean": float(iters[:, 0].mean()),
        "pcg_iters_per_rve_mean": float(iters[:, 1].mean()), "transfer_pcg_iters_per_rve_mean": float(iters[:, 2].mean()),
        "phase_ms": {"macro_qp_F": statistics.mean(ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)),
                     "rve_solve": statistics.mean(rve_ms),
                     "macro_assemble": statistics.mean(ev[k][2].elapsed_time(ev[k][3]) for k in range(args.steps)),
                     "macro_solve": statistics.mean(ev[k][3].elapsed_time(ev[k][4]) for k in range(args.steps))},
        "macro_cg_iters": int(info[1].item()),
        "roofline": {"kernel": f"rve{d}d_kernel<float>", "bound": "alu",
                     "achieved": ach_eq, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s (FP32-equivalent)",
                     "frac": ach_eq / FP32_PEAK_TFLOPS, "traffic": None,
                     "fp64_tflops": f64 / t_rve / 1e12, "fp32_tflops": f32 / t_rve / 1e12,
                     "note": "FP64 flops weighted by FP32/FP64 peak ratio; peaks from unit counts x 2.07 GHz"},
        "e2e": {"value": n_total / (statistics.median(e2e_ms) / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(budget_s, step_index=1):
    """The FP64 oracle as it stands, one process, on a bounded sample: the first qps of the
    same workload (same RVEs, same Fbar), solved until the time budget is spent."""
    from oracle.rve import PeriodicRVE
    p, Fload = build_problem(step_index)
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget_s and done < p.n_qp:
        r = p.qp_rve[done]
        PeriodicRVE(int(p.rve_n[r]), p.dim, p.rve_phase[r], p.rve_E[r], p.rve_nu[r]).solve(Fload, rtol=1e-10)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} of {p.n_qp} qps of the same workload (full Newton + tangent transfer, "
                      f"scipy sparse LU), {dt:.1f} s on one host core"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle.rve import PeriodicRVE
    p, Fload = build_problem(args.step_index)
    per_step = max(1, args.ref_rves_per_step)

    def step(k):
        for j in range(per_step):
            q = (k * per_step + j) % p.n_qp
            r = p.qp_rve[q]
            PeriodicRVE(int(p.rve_n[r]), p.dim, p.rve_phase[r], p.rve_E[r], p.rve_nu[r]).solve(Fload, rtol=1e-10)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator, config-2 shapes)", "config": workload_config(args.step_index),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} RVE solves of the workload per step (of {p.n_qp})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--step-index", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-rves-per-step", type=int, default=4)
    ap.add_argument("--cg-rtol", type=float, default=None, help="override the Newton-correction PCG tolerance")
    ap.add_argument("--cond-rtol", type=float, default=None, help="override the tangent-transfer PCG tolerance")
    ap.add_argument("--macro", type=int, default=None, help="macro elements per axis (profiling runs use less)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3"],
                    help="c2: 2D 4096 RVEs of 32x32 (default, the headline); c3: 3D 4096 uneven Hex8 RVEs")
    args = ap.parse_args()
    _SIZE["workload"] = args.workload
    _SIZE["macro"] = args.macro if args.macro is not None else (MACRO_C3 if args.workload == "c3" else MACRO)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
