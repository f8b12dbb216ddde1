"""Benchmark of the batched periodic-RVE hot path on one (or N) GB300.

Workload: the 2D plane-strain FE-HMM workload with a 32x32 Q1 macro mesh (4096 macro quadrature
points) and one 32x32 Q1 periodic RVE per point (random circular inclusion, stiffness ratio
5-50), mixed FP32/FP64 precision, loaded to biaxial 30% + shear 0.3 in 20 steps.  One timed
"step" is one whole load step of the nested scheme: macro iterations to macro convergence, each
Fbar at the quadrature points -> the batched RVE Newton solves with homogenised stress and
tangent -> macro residual/tangent assembly -> macro CG correction, starting from the converged
state of the previous load step.  The K timed steps cycle through load steps 1, 10 and 20 (the
states are reached by running the whole load path once before timing; it is reported too).

Value: RVE solves per second (whole job, all ranks).  Also reported: per-load-step rates,
micro-DOF x Newton iterations per second, the RVE kernel's ALU roofline fraction, parity of
P and A against the FP64 oracle at the GPU's own Fbar, and the oracle's rate on one and on all
host cores.  `--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead.  `--mode iteration` times macro iteration 1 of one load step from the zero
state (the short form used for profiling).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload c2|c3|...]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RVE solves/s (micro-DOF*Newton-iter/s reported alongside)"
_SIZE = {"macro": 32, "workload": "c2", "world": 1}
UNIT = "RVE solves/s"
MACRO, RVE_N, N_STEPS = 32, 32, 20
MACRO_C3, N_STEPS_C3 = 8, 10

# Algorithmic operation counts per unit of the 2D mixed kernel, counted from the kernel source
# (an FMA counting 2).
# residual: differences of the corner fluctuations (12), F's two columns at the two Gauss
# abscissae (32), per Gauss point J, the refined reciprocal (4 FMA), c and P (26 x 4), the stress
# sums per Gauss line and their shape weights (43), nodal forces (8), gather and norm (10)
FP64_FLOP_PER_ELEMENT_RESIDUAL = 211.0
FP32_FLOP_PER_ELEMENT_TANGENT = 1350.0   # 8x8 element tangent at 4 Gauss points + stencil gather
FP32_FLOP_PER_NODE_PCG_ITER = 100.0      # 9-block 2x2 stencil apply + vector updates + 2 dots
FP32_FLOP_PER_ELEMENT_TRANSFER = 1500.0  # energy form of the tangent transfer (4 unit gradients)
# multigrid preconditioner (2D, per fine node): V(1,1)-cycle per PCG iteration = two fine
# applies (2 x 72), smoothing, residuals, restriction and prolongation (180 on the fine level,
# 180/4 + 180/16 on the coarse levels, 2 for the coarsest 32 x 32 inverse apply); per tangent
# build the Galerkin coarse element matrices (748 FMA per coarse element: 374 + 94 + 23 per fine
# node), coarse stencils and the coarsest Gauss-Jordan inverse (2 x 32^3 / 1024)
FP32_FLOP_PER_NODE_MG_ITER = 238.0
FP32_FLOP_PER_NODE_MG_BUILD = 570.0
FP64_FLOP_PER_ELEMENT_RESIDUAL_3D = 2620.0   # Hex8: 8 Gauss points x (grad, cof(F), J, 1/J refined, P, nodal forces)
FP32_FLOP_PER_ELEMENT_TANGENT_3D = 4200.0    # Gauss-point data + 3x3 diagonal blocks
FP32_FLOP_PER_ELEMENT_APPLY_3D = 4000.0      # matrix-free apply: grad, dP = A:dF, nodal scatter
FP32_FLOP_PER_NODE_PCG_ITER_3D = 30.0        # preconditioner + vector updates + dots
# 3D multigrid, per fine element: V-cycle per PCG iteration = two more fine applies (2 x 4000),
# level-1 gathers (2 x 1152 flop per coarse node / 8), deeper levels, smoothing, restriction and
# prolongation; per tangent build the level-1 element blocks integrated over the 64 fine Gauss
# points of each coarse element (3312 flop per Gauss point, 212k per coarse element, 26.5k per
# fine element), deeper levels (2.3k) and the coarsest inverse (<= 0.6k)
FP32_FLOP_PER_ELEMENT_MG_ITER_3D = 8400.0
FP32_FLOP_PER_ELEMENT_MG_BUILD_3D = 29000.0
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
FP64_PEAK_TFLOPS = 1.25                              # GB300 nominal FP64


# DRAM bytes per RVE solve of the dominant kernel from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch / RVEs in that launch), with the profile summary it comes
# from; scaled to a launch of the bench by the RVEs it solves.  Only for a capture of the kernel
# build the bench runs: the captures in profiles/ (155 KB per 2D RVE, 23.9 MB per 3D RVE) predate
# the kernels' keeping of the coarse levels for the tangent transfer, so no entry is given.
TRAFFIC_PER_LAUNCH = {}


def workload_config(step_index):
    MACRO = _SIZE["macro"]
    if _SIZE["workload"] == "c3":
        return {"workload": f"3D FE-HMM macro {MACRO}^3 Hex8 ({MACRO ** 3 * 8} qps), one periodic Hex8 RVE per qp "
                            f"of 8^3/12^3/16^3 elements (uniform draw), 1-4 spheres (volume fraction 0.1-0.3, "
                            f"stiffness ratio 10), neo-Hookean, mixed FP32/FP64, uneven batch in one persistent "
                            f"launch, macro iteration 1 of load step {step_index}/{N_STEPS_C3} (uniaxial to 20%)",
                "n_qp": MACRO ** 3 * 8, "rve_grid": "8/12/16 mixed", "load_step": step_index,
                "l2": "flushed (256 MB write) between timed steps"}
    W = _SIZE["world"]
    cfg = {"workload": f"2D plane-strain FE-HMM macro {MACRO}x{MACRO * W} Q1 ({MACRO * MACRO * W * 4} qps), "
                       f"one {RVE_N}x{RVE_N} Q1 periodic RVE per qp (random circular inclusion r~U(0.15,0.35), "
                       f"E ratio log-U[5,50]), neo-Hookean, mixed FP32/FP64, macro iteration 1 of load step "
                       f"{step_index}/{N_STEPS} (biaxial 30% + shear 0.3)",
           "n_qp": MACRO * MACRO * W * 4, "rve_grid": RVE_N, "micro_dofs_per_rve": 2 * RVE_N * RVE_N,
           "load_step": step_index, "l2": "flushed (256 MB write) between timed steps"}
    if W > 1:
        cfg["parallelism"] = (f"dp{W}: macro elements in {W} contiguous blocks balanced by RVE dofs, one per rank; "
                              "all-reduce of f and K, macro solve on rank 0, broadcast of du")
    return cfg


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
        fd, self.path = tempfile.mkstemp(prefix="fehmm_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
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
        p = synth.uniaxial_3d_uneven(macro=_SIZE["macro"])
        F = np.diag([1.0 + 0.2 * step_index / N_STEPS_C3, 1.0, 1.0])
        return p, F
    p = synth.biaxial_shear_2d(macro=_SIZE["macro"], rve=RVE_N, macro_y=_SIZE["macro"] * _SIZE["world"])
    lam = step_index / N_STEPS
    F = np.eye(2) + lam * (p.extra["F_end"] - np.eye(2))
    return p, F


def macro_n(d):
    """Macro elements per axis: a square/cubic mesh, taller in y by the rank count (2D weak scaling)."""
    n = [_SIZE["macro"]] * d
    if d == 2:
        n[1] *= _SIZE["world"]
    return n


def macro_affine_u(F):
    """u = (F - I) X at the macro nodes (x fastest)."""
    d = F.shape[0]
    axes = [np.arange(m + 1) / m for m in macro_n(d)]
    X = np.stack(np.meshgrid(*axes, indexing="ij"), -1)
    X = X.transpose(*range(d - 1, -1, -1), d).reshape(-1, d)
    return (X @ (F - np.eye(d)).T).reshape(-1)


def mg3_levels(n):
    """Coarse levels of the 3D multigrid for grid n (0: block-Jacobi), as the kernel decides."""
    l, m = 0, n
    while m > 3 and m % 2 == 0:
        m //= 2
        l += 1
    return l if (m <= 3 and l >= 1) else 0


def flops_3d(p, iters, mg=False):
    """FP64 and FP32 algorithmic flops of one 3D batch solve from the per-qp iteration counts."""
    ns = np.array([int(p.rve_n[r]) for r in p.qp_rve])
    el = ns.astype(np.float64) ** 3
    on = np.array([mg and mg3_levels(int(n)) > 0 for n in ns], dtype=np.float64)
    newton = iters[:, 0].astype(np.float64)
    cg = iters[:, 1].astype(np.float64) + iters[:, 2].astype(np.float64)
    f64 = ((newton + 1) * FP64_FLOP_PER_ELEMENT_RESIDUAL_3D * el).sum()
    # the coarse levels are built at the first Newton iteration and for the tangent transfer
    f32 = ((newton + 1) * FP32_FLOP_PER_ELEMENT_TANGENT_3D * el + 2 * on * FP32_FLOP_PER_ELEMENT_MG_BUILD_3D * el
           + (cg + 9) * (FP32_FLOP_PER_ELEMENT_APPLY_3D + FP32_FLOP_PER_NODE_PCG_ITER_3D) * el
           + cg * on * FP32_FLOP_PER_ELEMENT_MG_ITER_3D * el).sum()
    return f64, f32


def flops_2d(n, iters, mg=False):
    """FP64 and FP32 algorithmic flops of one RVE batch solve from the per-qp iteration counts."""
    el = n * n
    newton = iters[:, 0].astype(np.float64)
    cg = iters[:, 1].astype(np.float64) + iters[:, 2].astype(np.float64)
    f64 = ((newton + 1) * FP64_FLOP_PER_ELEMENT_RESIDUAL * el).sum()
    per_iter = FP32_FLOP_PER_NODE_PCG_ITER + (FP32_FLOP_PER_NODE_MG_ITER if mg else 0.0)
    per_build = FP32_FLOP_PER_ELEMENT_TANGENT + (FP32_FLOP_PER_NODE_MG_BUILD if mg else 0.0)
    f32 = ((newton + 1) * per_build * el + cg * per_iter * el + FP32_FLOP_PER_ELEMENT_TRANSFER * el).sum()
    return f64, f32


TIMED_LOAD_STEPS = {"c2": (1, 10, 20), "c3": (1, 5, 10)}


def measured_peaks(dev):
    """cuBLAS DGEMM and SGEMM (TF32 off) rates on this GPU, measured live: the FP64 denominator of
    the ALU roofline and a cross-check of the FP32 unit-count peak."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in (("fp64_dgemm_tflops", torch.float64, 4096), ("fp32_sgemm_tflops", torch.float32, 8192)):
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            for _ in range(2):
                torch.matmul(a, b)
            torch.cuda.synchronize()
            best = 1e30
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    out["how"] = "torch.matmul (cuBLAS) float64 4096^3 and float32 8192^3 with TF32 off, best of 5, CUDA events"
    return out


def _oracle_rve(task):
    """One FP64 oracle RVE solve (module-level so that a spawned pool can run it)."""
    n, dim, phase, E, nu, F, rtol = task
    from oracle.rve import PeriodicRVE
    r = PeriodicRVE(n, dim, phase, E, nu).solve(F, rtol=rtol)
    return r["P"], r["A"]


def oracle_parity_and_baseline(p, F, P, A, qps, budget_s, label):
    """The FP64 oracle on one host core at the GPU's own Fbar of the given points (first ones, until
    the time budget is spent): per-point relative error of the GPU's P and A against it, and the
    oracle's rate.  Returns (parity dict, seconds, solves)."""
    d = p.dim
    t0 = time.perf_counter()
    eP, eA, done = [], [], 0
    for q in qps:
        if time.perf_counter() - t0 > budget_s and done >= (4 if p.dim == 2 else 1):
            break
        r = p.qp_rve[q]
        Pr, Ar = _oracle_rve((int(p.rve_n[r]), d, p.rve_phase[r], p.rve_E[r], p.rve_nu[r], F[q].reshape(d, d),
                              1e-12))
        eP.append(np.linalg.norm(P[q] - Pr.reshape(-1)) / max(np.linalg.norm(Pr), 1e-3))
        eA.append(np.linalg.norm(A[q] - Ar.reshape(-1)) / np.linalg.norm(Ar))
        done += 1
    dt = time.perf_counter() - t0
    return ({"state": label, "n": done, "max_rel_P": float(max(eP)), "max_rel_A": float(max(eA)),
             "tolerance": 1e-5}, dt, done)


def cpu_all_cores(p, F, qps, budget_s):
    """The oracle over a spawned process pool on every host core (one solve per task, BLAS
    threads pinned to 1): RVE solves/s on a bounded sample of the same points."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    d = p.dim
    tasks = []
    for q in qps:
        r = p.qp_rve[q]
        tasks.append((int(p.rve_n[r]), d, p.rve_phase[r], p.rve_E[r], p.rve_nu[r], F[q].reshape(d, d), 1e-10))
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_rve, tasks[:cores])  # start-up (imports) outside the timed part
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < budget_s and n < len(tasks):
            m = min(len(tasks) - n, cores * 2)
            pool.map(_oracle_rve, tasks[n:n + m])
            n += m
        dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} RVE solves (points of the bench's load-step-1 state, the GPU's own Fbar), "
                      f"{dt:.1f} s over a spawned pool of {cores} processes"}


def run_gpu(args):
    """Default mode: whole load steps of the load path.  A timed step is one complete load step
    (every macro iteration to macro convergence: Fbar, the batched RVE solves, assembly, macro
    CG, and the final accuracy pass) started from the converged state of the previous step; the
    K timed steps cycle through load steps TIMED_LOAD_STEPS (e.g. 1, 10 and 20 of 20).  The
    states are reached by running the load path once before timing."""
    import torch
    import torch.distributed as dist

    import paper_1908_08292_gb300 as fe
    from paper_1908_08292_gb300.driver import LoadStepDriver

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    wl = _SIZE["workload"]
    _SIZE["world"] = world if wl == "c2" else 1
    fe.lib()
    p, _ = build_problem(1)
    d = p.dim
    opts = {k: v for k, v in (("cg_rtol", args.cg_rtol), ("cond_rtol", args.cond_rtol)) if v is not None}
    opts["precond"] = fe.PRECOND_MG if args.precond == "mg" else fe.PRECOND_JACOBI
    shard = None
    if _SIZE["world"] > 1:
        from paper_1908_08292_gb300.dist import Shard
        dofs = np.array([d * int(p.rve_n[r]) ** d for r in p.qp_rve])
        shard = Shard.make(rank, world, dofs, 2 ** d)
    drv = LoadStepDriver(p, precision="mixed", shard=shard, predictor=True, **opts)
    ctx = drv.ctx
    steps_timed = TIMED_LOAD_STEPS[wl]
    n_total = p.n_qp if _SIZE["world"] > 1 else p.n_qp * world  # sharded mesh, or replicas
    mine = shard.qps if shard is not None else np.arange(p.n_qp)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    peaks = measured_peaks(dev)

    def ev():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # ---- the load path once (set-up, also reported); snapshots of the states the timed steps start from
    snaps, path = {}, []
    for k in range(1, max(steps_timed) + 1):
        if k in steps_timed:
            snaps[k] = drv.state()
        e0, e1 = ev()
        e0.record(stream)
        rec = drv.load_step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        path.append({"step": k, "ms": e0.elapsed_time(e1), "rve_passes": rec["rve_passes"],
                     "macro_iters": rec["macro_iters"], "converged": rec["converged"]})

    tuned, t_tune = None, 0.0
    if args.autotune == "on" or (args.autotune == "auto" and wl == "c3"):
        # the solver settings for the timed steps, timed on a sample of the points solving the
        # last load step of the path: from the fluctuations committed before it, at the macro
        # deformation it converged to (the snapshots do not depend on the settings)
        ctx.macro_qp_F(drv.u, drv.F)
        F_last = drv.F.clone()
        drv.restore(snaps[max(steps_timed)])
        t3 = time.perf_counter()
        tuned = ctx.autotune(F_last, n_sample=0)
        torch.cuda.synchronize()
        t_tune = time.perf_counter() - t3

    def restore(k):
        drv.restore(snaps[k])
        flush.zero_()

    for j in range(args.warmup):
        restore(steps_timed[j % len(steps_timed)])
        drv.load_step(steps_timed[j % len(steps_timed)], commit=False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launches
    recs = []
    with ClockSampler(local) as clk:
        for j in range(args.steps):
            k = steps_timed[j % len(steps_timed)]
            restore(k)
            drv.rve_events = []
            e0, e1 = ev()
            e0.record(stream)
            rec = drv.load_step(k, commit=False)
            e1.record(stream)
            torch.cuda.synchronize()
            recs.append({"k": k, "ms": e0.elapsed_time(e1), "passes": rec["rve_passes"],
                         "rve_ms": [a.elapsed_time(b) for a, b in drv.rve_events],
                         "macro_iters": rec["macro_iters"], "converged": rec["converged"]})
            drv.rve_events = None
    launches = ctx.launches - launches0
    if world > 1:
        dist.barrier()
    t_total = sum(r["ms"] for r in recs) / 1e3
    if world > 1:
        tt = torch.tensor([t_total], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total = float(tt.item())
    solves = sum(r["passes"] for r in recs) * n_total

    # ---- operation counts (untimed repetition of each timed load step; the 2D solves are
    # deterministic per point, the 3D ones up to the order of float atomics)
    counts = {}
    for k in steps_timed:
        restore(k)
        drv.iter_log = []
        drv.load_step(k, commit=False)
        its = [t.cpu().numpy()[mine] for t in drv.iter_log]
        drv.iter_log = None
        f64 = f32 = 0.0
        newton = cg = tr = 0.0
        for it in its:
            a, b = (flops_2d(RVE_N, it, args.precond == "mg") if d == 2 else flops_3d(p, it, args.precond == "mg"))
            f64 += a
            f32 += b
            newton += float(it[:, 0].mean())
            cg += float(it[:, 1].mean())
            tr += float(it[:, 2].mean())
        counts[k] = {"f64": f64, "f32": f32, "passes": len(its), "newton_per_rve_pass": newton / len(its),
                     "pcg_per_rve_pass": cg / len(its), "transfer_pcg_per_rve_pass": tr / len(its)}

    # ---- parity with the FP64 oracle at the GPU's own Fbar (final pass of load steps 1 and last)
    parity, cpu_one = [], None
    for k in (steps_timed[0], steps_timed[-1]):
        restore(k)
        drv.load_step(k, commit=False)
        torch.cuda.synchronize()
        Fh, Ph, Ah = drv.F.cpu().numpy(), drv.P.cpu().numpy(), drv.A.cpu().numpy()
        if rank == 0 and not args.no_cpu_baseline:
            budget = args.cpu_seconds if k == steps_timed[0] else args.cpu_seconds / 3
            par, dt, n = oracle_parity_and_baseline(p, Fh, Ph, Ah, mine, budget, f"load step {k}, final pass")
            parity.append(par)
            if k == steps_timed[0]:
                cpu_one = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                           "sample": f"first {n} of {p.n_qp} points at the GPU's Fbar of load step {k} (final "
                                     f"pass), full Newton + tangent transfer, scipy sparse LU, {dt:.1f} s on one "
                                     f"host core"}
                F_state1 = Fh

    # ---- end to end through the public API with host buffers (H2D of u, D2H of u, P, A, status)
    u_h = torch.empty_like(drv.u, device="cpu").pin_memory()
    outs_h = [torch.empty_like(t, device="cpu").pin_memory() for t in (drv.u, drv.P, drv.A, drv.st)]
    e2e_s, e2e_solves = 0.0, 0
    for j in range(max(1, args.steps)):
        k = steps_timed[j % len(steps_timed)]
        restore(k)
        u_h.copy_(snaps[k][0])  # the macro state of the step's start, staged in pinned host memory
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        drv.u.copy_(u_h, non_blocking=True)
        rec = drv.load_step(k, commit=False)
        for h, t in zip(outs_h, (drv.u, drv.P, drv.A, drv.st)):
            h.copy_(t, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        e2e_solves += rec["rve_passes"] * n_total
    h2d = u_h.numel() * 8
    d2h = sum(h.numel() * h.element_size() for h in outs_h)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    value = solves / t_total
    per_step = {}
    for k in steps_timed:
        rs = [r for r in recs if r["k"] == k]
        if rs:
            t = sum(r["ms"] for r in rs) / 1e3
            per_step[str(k)] = {"rve_solves_per_s": sum(r["passes"] for r in rs) * n_total / t,
                                "ms_per_load_step": 1e3 * t / len(rs), "macro_iters": rs[0]["macro_iters"],
                                "rve_passes": rs[0]["passes"], **{kk: v for kk, v in counts[k].items()
                                                                  if kk not in ("f64", "f32", "passes")}}
    # dominant kernel: the batched RVE solve; achieved = algorithmic flops per launch / mean launch time
    rve_ms = [m for r in recs for m in r["rve_ms"]]
    n_launch = len(rve_ms)
    f64 = sum(counts[r["k"]]["f64"] for r in recs)
    f32 = sum(counts[r["k"]]["f32"] for r in recs)
    t_launch = statistics.mean(rve_ms) / 1e3
    fp64_peak = peaks["fp64_dgemm_tflops"]
    ach_eq = (f32 + f64 * FP32_PEAK_TFLOPS / fp64_peak) / n_launch / t_launch / 1e12
    dofs = np.array([d * int(p.rve_n[r]) ** d for r in p.qp_rve[mine]], dtype=np.float64)
    dof_iter = sum(counts[r["k"]]["newton_per_rve_pass"] * counts[r["k"]]["passes"] for r in recs) \
        * float(dofs.mean()) * n_total / t_total
    traffic = TRAFFIC_PER_LAUNCH.get((wl, args.precond))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed: FP64 residual/sums, FP32 tangent/PCG)",
        "data": "synthetic (seeded generator, config shapes)", "config": path_config(steps_timed),
        "micro_dof_newton_iter_per_s": dof_iter,
        "rve_preconditioner": ("multigrid V(1,1) with Galerkin coarse levels" if args.precond == "mg"
                               else "block-Jacobi"),
        "timed_steps_converged": all(r["converged"] for r in recs),
        "autotuned": ({"choice": tuned, "seconds": t_tune} if tuned is not None else None),
        "per_load_step": per_step,
        "load_path": {"steps": len(path), "seconds": sum(x["ms"] for x in path) / 1e3,
                      "rve_solves": sum(x["rve_passes"] for x in path) * n_total,
                      "rve_solves_per_s": sum(x["rve_passes"] for x in path) * n_total / (sum(x["ms"] for x in path) / 1e3),
                      "macro_iters_per_step": [x["macro_iters"] for x in path],
                      "all_converged": all(x["converged"] for x in path),
                      "note": "the whole load path once, before timing (includes first-use costs)"},
        "roofline": {"kernel": f"rve{d}d_kernel<float>", "bound": "alu",
                     "achieved": ach_eq, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s (FP32-equivalent)",
                     "frac": ach_eq / FP32_PEAK_TFLOPS,
                     "traffic": traffic[0] * (n_total / world) if traffic else None,
                     "traffic_source": traffic[1] if traffic else None,
                     "launches": n_launch, "mean_launch_ms": t_launch * 1e3,
                     "fp64_tflops": f64 / n_launch / t_launch / 1e12, "fp32_tflops": f32 / n_launch / t_launch / 1e12,
                     "note": "FP32 peak from unit counts (152 SMs x 128 lanes x 2 x 2.07 GHz); FP64 flops weighted "
                             "by FP32 peak / measured DGEMM rate; flops counted from the kernel source per unit "
                             "x the per-point iteration counts of each launch"},
        "peaks_measured": peaks,
        "parity": parity,
        "e2e": {"value": e2e_solves / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_one
        out["cpu_baseline_all_cores"] = cpu_all_cores(p, F_state1, mine[: 64 * (os.cpu_count() or 1)],
                                                      args.cpu_seconds / 2)
    drv.close()
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def path_config(steps_timed):
    wl = _SIZE["workload"]
    W = _SIZE["world"]
    MACRO = _SIZE["macro"]
    ks = ", ".join(str(k) for k in steps_timed)
    if wl == "c3":
        return {"workload": f"3D FE-HMM macro {MACRO}^3 Hex8 ({MACRO ** 3 * 8} qps), one periodic Hex8 RVE per qp "
                            f"of 8^3/12^3/16^3 elements (uniform draw), 1-4 spheres (volume fraction 0.1-0.3, "
                            f"stiffness ratio 10), neo-Hookean, mixed FP32/FP64, uneven batch in one persistent "
                            f"launch; a step = one whole load step (all macro iterations, nested scheme) of the "
                            f"10-step uniaxial path to 20%, cycling load steps {ks}",
                "n_qp": MACRO ** 3 * 8, "rve_grid": "8/12/16 mixed", "load_steps_timed": list(steps_timed),
                "l2": "flushed (256 MB write) between timed steps"}
    cfg = {"workload": f"2D plane-strain FE-HMM macro {MACRO}x{MACRO * W} Q1 ({MACRO * MACRO * W * 4} qps), "
                       f"one {RVE_N}x{RVE_N} Q1 periodic RVE per qp (random circular inclusion r~U(0.15,0.35), "
                       f"E ratio log-U[5,50]), neo-Hookean, mixed FP32/FP64; a step = one whole load step (all "
                       f"macro iterations to convergence, nested scheme, from the previous step's converged "
                       f"state) of the 20-step path to biaxial 30% + shear 0.3, cycling load steps {ks}",
           "n_qp": MACRO * MACRO * W * 4, "rve_grid": RVE_N, "micro_dofs_per_rve": 2 * RVE_N * RVE_N,
           "load_steps_timed": list(steps_timed), "l2": "flushed (256 MB write) between timed steps"}
    if W > 1:
        cfg["parallelism"] = (f"dp{W}: macro elements in {W} contiguous blocks balanced by RVE dofs, one per rank; "
                              "all-reduce of f and K, macro solve on rank 0, broadcast of du")
    return cfg


def run_gpu_iteration(args):
    """--mode iteration: macro iteration 1 of load step --step-index from the committed (zero)
    state with an affine macro field, repeated (profiling runs use this short form)."""
    import torch
    import torch.distributed as dist

    import paper_1908_08292_gb300 as fe

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    _SIZE["world"] = world if _SIZE["workload"] == "c2" else 1
    fe.lib()
    p, Fload = build_problem(args.step_index)
    n_qp = p.n_qp
    opts = {k: v for k, v in (("cg_rtol", args.cg_rtol), ("cond_rtol", args.cond_rtol)) if v is not None}
    opts["precond"] = fe.PRECOND_MG if args.precond == "mg" else fe.PRECOND_JACOBI
    d = p.dim
    ctx = fe.Context(d, "mixed", **opts)
    ctx.add_rves(p.rve_n, p.rve_phase, p.rve_E, p.rve_nu)
    ctx.bind_qps(p.qp_rve)
    ctx.macro_create(macro_n(d))
    ctx.macro_set_dirichlet(p.dirichlet_dofs, p.dirichlet_end)
    _, _, n_rows, nnz = ctx.macro_csr()
    u_h = torch.tensor(macro_affine_u(Fload), dtype=torch.float64).pin_memory()
    u = u_h.to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    if _SIZE["world"] > 1:
        # weak scaling: the macro mesh is `world` times taller, each rank solves the RVEs of its
        # contiguous block of macro elements; one sum of f and K per iteration, rank 0 solves
        from paper_1908_08292_gb300.dist import Shard, ShardedIteration
        dofs = np.array([d * int(p.rve_n[r]) ** d for r in p.qp_rve])
        shard = Shard.make(rank, world, dofs, 2 ** d)
        sit = ShardedIteration(ctx, shard, n_qp, d, dev)
        F, P, A, st, it, f, K, du, info = sit.F, sit.P, sit.A, sit.st, sit.it, sit.f, sit.K, sit.du, sit.info
        mine = shard.qps.astype(np.int64)

        def rve_phase():
            ctx.rve_solve_list(F, P, A, st, it, fe.SOLVE_FROM_COMMITTED, sit.lst, sit.cnt)

        def assemble_phase():
            ctx.macro_assemble(P, A, f, K)
            shard.reduce_system(f, K)

        def solve_phase():
            if rank == 0:
                ctx.macro_solve(K, f, du, info, rtol=1e-10)
            shard.share_correction(du)
    else:
        F = torch.empty(n_qp, d * d, dtype=torch.float64, device=dev)
        P = torch.empty(n_qp, d * d, dtype=torch.float64, device=dev)
        A = torch.empty(n_qp, d ** 4, dtype=torch.float64, device=dev)
        st = torch.empty(n_qp, dtype=torch.int32, device=dev)
        it = torch.empty(n_qp, 4, dtype=torch.int32, device=dev)
        f = torch.empty(n_rows, dtype=torch.float64, device=dev)
        K = torch.empty(nnz, dtype=torch.float64, device=dev)
        du = torch.empty(n_rows, dtype=torch.float64, device=dev)
        info = torch.empty(3, dtype=torch.float64, device=dev)
        mine = np.arange(n_qp)

        def rve_phase():
            ctx.rve_solve(F, P, A, st, it, flags=fe.SOLVE_FROM_COMMITTED)

        def assemble_phase():
            ctx.macro_assemble(P, A, f, K)

        def solve_phase():
            ctx.macro_solve(K, f, du, info, rtol=1e-10)

    def step():
        ctx.macro_qp_F(u, F)
        rve_phase()
        assemble_phase()
        solve_phase()

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
            rve_phase()
            e2.record(stream)
            assemble_phase()
            e3.record(stream)
            solve_phase()
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
    status = st.cpu().numpy()[mine]
    iters = it.cpu().numpy()[mine]
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
    n_total = n_qp if _SIZE["world"] > 1 else n_qp * world  # sharded mesh, or one replica per rank
    value = n_total / (t_step / args.steps)
    dofs = np.array([d * int(p.rve_n[r]) ** d for r in p.qp_rve[mine]], dtype=np.float64)
    dof_iter = float((dofs * iters[:, 0].astype(np.float64)).sum()) * world / (t_step / args.steps)
    f64, f32 = (flops_2d(RVE_N, iters, args.precond == "mg") if d == 2
                else flops_3d(p, iters, args.precond == "mg"))
    t_rve = statistics.mean(rve_ms) / 1e3
    ach_eq = (f32 + f64 * FP32_PEAK_TFLOPS / FP64_PEAK_TFLOPS) / t_rve / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (mixed: FP64 residual/sums, FP32 tangent/PCG)",
        "data": "synthetic (seeded generator, the 2D 4096-RVE workload's shapes)", "config": workload_config(args.step_index),
        "micro_dof_newton_iter_per_s": dof_iter,
        "rve_preconditioner": ("multigrid V(1,1) with Galerkin coarse levels" if args.precond == "mg"
                               else "block-Jacobi"),
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
    """The FP64 oracle as it stands on one host core, on the arm's workload: each step solves
    --ref-rves-per-step points at the affine Fbar of the load steps the GPU arm times (cycling),
    from zero fluctuations (bounded sample; the oracle has no batch or load-path state)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle.rve import PeriodicRVE
    p, _ = build_problem(1)
    steps_timed = TIMED_LOAD_STEPS.get(_SIZE["workload"], (args.step_index,)) if args.mode == "path" else (args.step_index,)
    per_step = max(1, args.ref_rves_per_step)
    F_of = {ls: build_problem(ls)[1] for ls in steps_timed}

    def step(k):
        F = F_of[steps_timed[k % len(steps_timed)]]
        for j in range(per_step):
            q = (k * per_step + j) % p.n_qp
            r = p.qp_rve[q]
            PeriodicRVE(int(p.rve_n[r]), p.dim, p.rve_phase[r], p.rve_E[r], p.rve_nu[r]).solve(F, rtol=1e-10)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    cfg = path_config(steps_timed) if args.mode == "path" else workload_config(args.step_index)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator, config shapes)", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} RVE solves per step at the affine Fbar of load steps "
                                   f"{list(steps_timed)} (cycling), from zero fluctuations (of {p.n_qp} points)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _u_ball_problem(macro):
    """The large 3D macro problem of the surrogate comparison (macro^3 Hex8, the fixed 12^3 RVE at every point)."""
    import synth
    return synth.cantilever_3d_fixed_rve(macro=macro)


def _heldout_oracle():
    """The stored FP64 oracle values of the surrogate workload's held-out set (tests/golden/c4_heldout_oracle.txt,
    written by tests/golden/make_c4_heldout.py from oracle/ only): {q: (status, P[9], W)}."""
    path = os.path.join(ROOT, "tests", "golden", "c4_heldout_oracle.txt")
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out[int(f[0])] = (int(f[1]), np.array([float(v) for v in f[3:12]]), float(f[12]))
    return out


def run_c4(args):
    """Surrogate training workload (c4): GPU RVE solves at U uniform in |U - I| <= 0.3 on the
    fixed 12^3 two-inclusion RVE (training targets), training with the library's BF16 kernels, and
    the held-out stress error: against the GPU RVE solves of the whole held-out set and against the
    stored FP64 oracle values of its first points; by stretch radius, with the largest trust radius
    whose held-out points all meet 1e-4."""
    import torch

    import synth
    from paper_1908_08292_gb300 import surrogate as su
    torch.cuda.set_device(0)
    one = su.fixed_rve_context(1)
    lam0, mu0, Ca = su.base_law(one)
    sp = su.SurrogateParams(lam0, mu0, 0.35, 0.01 * (lam0 + 2 * mu0), 0.3)
    sp.set_Ca(Ca)
    ctx = su.fixed_rve_context(4096)
    U = synth.stretch_ball(1004, args.c4_samples, 0.3)
    Uh = synth.stretch_ball(2004, args.c4_holdout, 0.3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, ty, tg, P, W, dropped = su.generate(ctx, sp, U)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    _, _, _, Ph, Wh, dropped_h = su.generate(ctx, sp, Uh, drop_failed=False)
    t_fit = 0.0
    if args.c4_poly:  # the polynomial part first; the network learns what it leaves
        t3 = time.perf_counter()
        su.fit_poly(sp, x, ty, tg, max_degree=args.c4_poly)
        torch.cuda.synchronize()
        t_fit = time.perf_counter() - t3
    mlp = su.MLP(4096)
    mlp.set_params(su.init_params(7, out_scale=args.c4_out_scale))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = su.train(mlp, x, ty, tg, args.c4_epochs, batch=4096, lr=args.c4_lr, lr_end=args.c4_lr / 100)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    steps = args.c4_epochs * (x.shape[0] // 4096)
    # the learned correction vanishes to third order at E = 0, where the base law carries the
    # RVE's exact small-strain tangent
    sp.set_origin(mlp, hessian=args.c4_hessian_origin)
    n = Uh.shape[0]
    Fh = torch.tensor(Uh.reshape(n, 9), device="cuda")
    Ps = torch.zeros(n, 9, dtype=torch.float64, device="cuda")
    As = torch.zeros(n, 81, dtype=torch.float64, device="cuda")
    ins = torch.zeros(n, dtype=torch.int32, device="cuda")
    m2 = su.MLP(n)
    m2.set_params(mlp.get_params())
    work = torch.zeros(su.work_floats(n), dtype=torch.float32, device="cuda")
    su.surrogate_eval(m2, sp, Fh, Ps, As, None, ins, work)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    su.surrogate_eval(m2, sp, Fh, Ps, As, None, ins, work)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t2
    Psn, Phn = Ps.cpu().numpy(), Ph.cpu().numpy()
    e = su.stress_errors(Psn, Phn, 1e-3)
    # the base law with the polynomial part alone (a zero network, no origin shift)
    sp0 = su.SurrogateParams.from_buffer_copy(sp)
    sp0.y0 = 0.0
    for k in range(6):
        sp0.g0[k] = 0.0
    for k in range(36):
        sp0.H0[k] = 0.0
    m2.set_params(np.zeros(su.n_params(), dtype=np.float32))
    su.surrogate_eval(m2, sp0, Fh, Ps, As, None, ins, work)
    e_base = su.stress_errors(Ps.cpu().numpy(), Phn, 1e-3)
    rad = np.linalg.norm((Uh - np.eye(3)).reshape(n, 9), axis=1)
    bins = {}
    for lo, hi in ((0.0, 0.05), (0.05, 0.1), (0.1, 0.15), (0.15, 0.2), (0.2, 0.25), (0.25, 0.3001)):
        m = (rad >= lo) & (rad < hi)
        if m.any():
            bins[f"{lo:.2f}-{min(hi, 0.3):.2f}"] = {"n": int(m.sum()), "rms": float(np.sqrt((e[m] ** 2).mean())),
                                                    "max": float(e[m].max())}
    order = np.argsort(rad)
    run_max = np.maximum.accumulate(e[order])
    ok = np.nonzero(run_max <= 1e-4)[0]
    r_star = float(rad[order][ok[-1]]) if ok.size else 0.0
    # the stored FP64 oracle values of the first held-out points: the GPU RVE solves and the surrogate
    ref = _heldout_oracle()
    qs = [q for q in sorted(ref) if q < n and ref[q][0] == 0]
    verified = {}
    if qs:
        Pref = np.stack([ref[q][1] for q in qs])
        e_rve = su.stress_errors(Phn[qs], Pref, 1e-3)
        e_sur = su.stress_errors(Psn[qs], Pref, 1e-3)
        verified = {"n": len(qs), "gpu_rve_vs_oracle_max": float(e_rve.max()),
                    "surrogate_vs_oracle_rms": float(np.sqrt((e_sur ** 2).mean())),
                    "surrogate_vs_oracle_max": float(e_sur.max()),
                    "source": "tests/golden/c4_heldout_oracle.txt (make_c4_heldout.py, oracle/ only)"}
    if args.c4_save:
        su.save(mlp, sp, args.c4_save)
    print(json.dumps({
        "metric": "surrogate training: RVE solves/s for training data; held-out relative stress error",
        "value": x.shape[0] / t_data, "unit": "RVE solves/s (12^3, 3-stage continuation)", "n_gpus": 1,
        "higher_is_better": True, "workload": "c4",
        "config": {"workload": f"fixed 12^3 two-inclusion RVE (ratio 10), {args.c4_samples} training U in "
                               f"|U-I|_F<=0.3, {args.c4_holdout} held-out, MLP 6-4x128 SiLU-1 BF16/FP32, AdamW "
                               f"batch 4096, {args.c4_epochs} epochs, lr {args.c4_lr:g} cosine to 1/100, output layer "
                               f"initialised x{args.c4_out_scale}, "
                               f"Sobolev loss (W and S), origin shift to "
                               f"{'third' if args.c4_hessian_origin else 'second'} order"
                               + (f", polynomial part of degree 3-{args.c4_poly} fitted first" if args.c4_poly else "")},
        "dropped_failed_solves": dropped + dropped_h, "base_law": {"lam0": lam0, "mu0": mu0},
        "train_seconds": t_train, "train_steps_per_s": steps / t_train, "loss_first_last": [hist[0], hist[-1]],
        "heldout_stress_err": {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max()),
                               "median": float(np.median(e)), "n": int(n), "by_radius": bins},
        "heldout_err_without_network": {"rms": float(np.sqrt((e_base ** 2).mean())), "max": float(e_base.max()),
                                        "what": "base law" + (" + polynomial part" if args.c4_poly else "")},
        "poly_fit_seconds": t_fit,
        "largest_radius_meeting_1e-4": r_star,
        "inference_points_per_s": n / t_inf, "oracle_verified": verified,
        "target_1e-4_met": bool(e.max() <= 1e-4),
    }))


def run_c5(args):
    """Surrogate comparison (c5): one macro iteration of the surrogate-with-fallback path vs the plain GPU RVE path
    from the same macro state (macro^3 Hex8, the fixed 12^3 RVE everywhere).  The surrogate
    iteration is timed in the state its own load path left (fallback points solve from whatever
    fluctuations they last committed); the plain iteration is timed after every point's RVE has
    been solved and committed at the previous load step's converged macro state, the warm start a
    plain run of the load path would have."""
    import torch

    import synth
    from paper_1908_08292_gb300 import SOLVE_FROM_COMMITTED
    from paper_1908_08292_gb300 import surrogate as su
    torch.cuda.set_device(0)
    mlp = su.MLP(max(4096, args.macro ** 3 * 8))
    if args.c4_load:  # the surrogate trained and saved by the c4 workload
        sp = su.load(mlp, args.c4_load)
        sp.radius = args.c5_radius
    else:
        one = su.fixed_rve_context(1)
        lam0, mu0, Ca = su.base_law(one)
        sp = su.SurrogateParams(lam0, mu0, 0.35, 0.01 * (lam0 + 2 * mu0), args.c5_radius)
        sp.set_Ca(Ca)
        gen = su.fixed_rve_context(4096)
        x, ty, tg, _, _, _ = su.generate(gen, sp, synth.stretch_ball(1004, args.c4_samples, 0.3))
        if args.c4_poly:
            su.fit_poly(sp, x, ty, tg, max_degree=args.c4_poly)
        mlp.set_params(su.init_params(7, out_scale=args.c4_out_scale))
        su.train(mlp, x, ty, tg, args.c4_epochs, batch=4096, lr=args.c4_lr, lr_end=args.c4_lr / 100)
        sp.set_origin(mlp, hessian=args.c4_hessian_origin)
        gen.close()
    p = _u_ball_problem(args.macro)
    drv = su.SurrogateDriver(p, mlp, sp, audit_stride=args.c5_audit_stride, precision="mixed", newton_rtol=1e-8)
    d = drv.drv
    for k in range(1, args.c5_step):  # reach the state of load step c5_step with the surrogate path
        d.load_step(k)
    u_prev = d.u.clone()  # the converged macro state of load step c5_step - 1
    d.scale = args.c5_step / p.n_steps
    d.ctx.macro_apply_dirichlet(d.u, d.du, d.scale)
    n = p.n_qp
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def surrogate_iteration():
        d.ctx.macro_qp_F(d.u, d.F)
        drv._constitutive(True)
        d.ctx.macro_assemble(d.P, d.A, d.f, d.K)
        d.ctx.macro_solve(d.K, d.f, d.du, d.info, rtol=1e-10)

    def plain_iteration():
        d.ctx.macro_qp_F(d.u, d.F)
        d.ctx.rve_solve(d.F, d.P, d.A, d.st, d.it, flags=SOLVE_FROM_COMMITTED)
        d.ctx.macro_assemble(d.P, d.A, d.f, d.K)
        d.ctx.macro_solve(d.K, d.f, d.du, d.info, rtol=1e-10)

    surrogate_iteration()  # warm-up
    t_s = min(timed(surrogate_iteration) for _ in range(max(1, args.steps)))
    fallback = drv.fallback_count()
    audit = drv.audit_errors(1e-3) if args.c5_audit_stride else np.zeros(0)
    P_sur = d.P.clone()
    # warm start of the plain path: RVE solves at the previous step's converged state, committed
    F_prev = torch.zeros_like(d.F)
    d.ctx.macro_qp_F(u_prev, F_prev)
    d.ctx.rve_solve(F_prev, d.P, d.A, d.st, d.it, flags=SOLVE_FROM_COMMITTED)  # also keeps transfer solutions
    primed_ok = int((d.st.cpu().numpy() <= 1).sum())
    d.ctx.commit()
    t_p = timed(plain_iteration)
    st = d.st.cpu().numpy()
    e = su.stress_errors(P_sur.cpu().numpy(), d.P.cpu().numpy(), 1e-3)
    print(json.dumps({
        "metric": "macro Newton iterations/s, surrogate+fallback vs plain GPU RVE path",
        "value": 1.0 / t_s, "unit": "macro iterations/s", "n_gpus": 1, "higher_is_better": True,
        "workload": "c5",
        "config": {"workload": f"macro {args.macro}^3 Hex8 ({n} qps), fixed 12^3 two-inclusion RVE at every qp, "
                               f"clamped at x=0, shear+tension to |F-I|=0.35 in {p.n_steps} steps; state of load "
                               f"step {args.c5_step}; trust radius {args.c5_radius}"},
        "plain_value": 1.0 / t_p, "gain": t_p / t_s, "seconds": {"surrogate": t_s, "plain": t_p},
        "fallback_points": fallback, "fallback_fraction": fallback / n, "plain_status_ok": int((st == 0).sum()),
        "plain_warm_start": {"what": "every RVE solved (with its tangent transfer) and committed at load step "
                                     "c5_step - 1's converged state before the plain iteration is timed",
                             "points_ok": primed_ok},
        "audit": {"n": int(audit.size), "rms": float(np.sqrt((audit ** 2).mean())) if audit.size else None,
                  "max": float(audit.max()) if audit.size else None},
        "stress_err_vs_plain": {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max())},
        "target_1e-4_met": bool(e.max() <= 1e-4),
    }))


def run_mlp(args):
    """The surrogate network's kernels alone: AdamW training steps (loss, exact parameter gradient
    of the Sobolev loss, update) at batch 4096 and the inference pass the surrogate evaluation runs
    (value, input gradient and input Hessian) over a c5-sized set of points, each timed with CUDA
    events on the launching stream over --steps repetitions after --warmup.  The 128 x 128 layer
    products run on tcgen05; `gemm_tflops` divides their flops by the whole call's time (a lower
    bound of the products' own rate)."""
    import torch

    import synth
    from paper_1908_08292_gb300 import surrogate as su
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    B, n_inf = 4096, args.mlp_points
    m = su.MLP(max(B, n_inf))
    m.set_params(su.init_params(7))
    x = torch.tensor(synth.random_field(81, n_inf, 6, 0.9), dtype=torch.float32, device=dev)
    ty = torch.tensor(synth.random_field(82, 1, B, 1.0)[0], dtype=torch.float32, device=dev)
    tg = torch.tensor(synth.random_field(83, B, 6, 1.0), dtype=torch.float32, device=dev)
    y = torch.zeros(n_inf, dtype=torch.float32, device=dev)
    g = torch.zeros(n_inf, 6, dtype=torch.float32, device=dev)
    H = torch.zeros(n_inf, 6, 6, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def train_step():
        m.loss_grad(x[:B], ty, tg, 1.0 / B, 1.0 / B, loss)
        m.adamw(1e-4)

    def infer():
        m.eval(x, y, g, H)

    def timed(fn, reps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = m.launches()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps, (m.launches() - l0) // reps

    t_train, l_train = timed(train_step, args.steps)
    t_inf, l_inf = timed(infer, args.steps)
    m.check()
    sq = 2.0 * 128 * 128
    f_train = 18 * B * sq       # 128 x 128 products per training step
    f_inf = (6 + 36) * n_inf * sq  # forward + backward (B rows) and 6 tangent directions (6B rows)
    print(json.dumps({
        "metric": "surrogate network: AdamW training steps/s (batch 4096) and inference points/s",
        "value": 1.0 / t_train, "unit": "training steps/s", "workload": "mlp", "n_gpus": 1,
        "higher_is_better": True, "dtype": "bf16 operands, f32 accumulation",
        "config": {"workload": f"MLP 6-4x128 SiLU-1, training batch {B}, inference {n_inf} points with "
                               f"input gradient and Hessian", "steps": args.steps},
        "train_ms": t_train * 1e3, "train_launches": int(l_train),
        "train_gemm_tflops_lower_bound": f_train / t_train / 1e12,
        "inference_points_per_s": n_inf / t_inf, "inference_ms": t_inf * 1e3, "inference_launches": int(l_inf),
        "inference_gemm_tflops_lower_bound": f_inf / t_inf / 1e12,
    }))


def run_hconv(args):
    """Micro mesh convergence (the a-priori estimates of Sec. 4, the micro-convergence studies of
    Sec. 6): one microstructure, a box inclusion [0.25, 0.75)^d of stiffness ratio 10 that every
    grid n = 4, 8, ... resolves exactly, solved on the GPU in FP64 at a finite-strain Fbar with
    periodic and with KUBC coupling; relative errors of Pbar and Abar against the finest grid and
    the observed orders.  Also the modelling error of KUBC (Eq. ModelingError): the KUBC-periodic
    gap of Abar on k x k tilings of one cell, and the macro displacement of the 4x4 Q1 uniaxial problem
    computed with RVE grids 8, 16, 32 of the same microstructure."""
    import dataclasses

    import torch

    import paper_1908_08292_gb300 as fe
    import synth
    from paper_1908_08292_gb300.driver import LoadStepDriver
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    strict = dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-9, cond_rtol=1e-12)
    Fs = {2: np.array([[1.12, 0.06], [0.03, 0.95]]),
          3: np.array([[1.10, 0.05, 0.0], [0.02, 0.96, 0.03], [0.0, 0.01, 0.97]])}
    grids = {2: [4, 8, 16, 32], 3: [4, 8, 16]}

    def batch(dim, ns, phases, bc):
        n_q = len(ns)
        with fe.Context(dim, "fp64", bc=bc, **strict) as ctx:
            ctx.add_rves(ns, phases, [[1.0, 10.0]] * n_q, [[0.3, 0.3]] * n_q)
            ctx.bind_qps(np.arange(n_q, dtype=np.int32))
            F = torch.tensor(np.stack([Fs[dim]] * n_q).reshape(n_q, -1), dtype=torch.float64, device=dev)
            P = torch.zeros(n_q, dim * dim, dtype=torch.float64, device=dev)
            A = torch.zeros(n_q, dim ** 4, dtype=torch.float64, device=dev)
            st = torch.zeros(n_q, dtype=torch.int32, device=dev)
            ctx.rve_solve(F, P, A, st)
            torch.cuda.synchronize()
            assert (st.cpu().numpy() == 0).all()
            return P.cpu().numpy(), A.cpu().numpy()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    out = {"metric": "micro h-convergence of Pbar and Abar; KUBC modelling error; macro u vs RVE grid",
           "workload": "hconv", "n_gpus": 1, "unit": "relative error", "higher_is_better": False, "studies": []}
    for dim in (2, 3):
        ns = grids[dim]
        for bc, name in ((0, "periodic"), (1, "KUBC")):
            P, A = batch(dim, ns, [synth.box_inclusion(n, dim) for n in ns], bc)
            eP = [rel(P[k], P[-1]) for k in range(len(ns) - 1)]
            eA = [rel(A[k], A[-1]) for k in range(len(ns) - 1)]
            out["studies"].append({"dim": dim, "coupling": name, "grids": ns, "reference": ns[-1],
                                   "err_P": eP, "err_A": eA,
                                   "order_A": [float(np.log2(eA[k] / eA[k + 1])) for k in range(len(eA) - 1)]})
    # KUBC modelling error: k x k tilings of the 8 x 8 cell (the periodic result is tiling-invariant)
    ks = [1, 2, 4]
    tiles = [np.tile(synth.box_inclusion(8, 2).reshape(8, 8), (k, k)).reshape(-1) for k in ks]
    _, Ap = batch(2, [8 * k for k in ks], tiles, 0)
    _, Ak = batch(2, [8 * k for k in ks], tiles, 1)
    out["kubc_gap"] = {"tilings": ks, "gap_A": [rel(Ak[j], Ap[j]) for j in range(len(ks))],
                       "periodic_tiling_invariance": [rel(Ap[j], Ap[0]) for j in range(len(ks))]}
    # the 4x4 Q1 uniaxial macro problem with RVE grids 8, 16, 32 of the box microstructure
    base = synth.uniaxial_2d_small()
    us = {}
    for n in (8, 16, 32):
        p = dataclasses.replace(base, rve_n=np.array([n]), rve_phase=[synth.box_inclusion(n, 2)])
        drv = LoadStepDriver(p, precision="fp64", newton_rtol=1e-12, newton_atol=1e-15, cg_rtol=1e-9, cond_rtol=1e-11)
        try:
            for k in range(1, p.n_steps + 1):
                assert drv.load_step(k)["converged"]
            us[n] = drv.u.cpu().numpy()
        finally:
            drv.close()
    out["macro_u"] = {"rve_grids": [8, 16], "reference": 32,
                      "err_u": [rel(us[n], us[32]) for n in (8, 16)]}
    print(json.dumps(out))


def run_schemes(args):
    """Algorithm 1 (nested) vs Algorithm 2 (alternating) on full load paths: macro iterations,
    micro Newton iterations and wall time per scheme (the structure of the paper's speed-up
    tables; synthetic microstructures stand in for the paper's)."""
    import torch

    import synth
    from paper_1908_08292_gb300.driver import LoadStepDriver
    torch.cuda.set_device(0)
    cases = [("c1 2D 4x4 Q1 macro, 64 qps, 8x8 RVE (FP64), 10 steps", synth.uniaxial_2d_small(), 10, {}),
             ("c2-shaped 2D 8x8 Q1 macro, 256 qps, 32x32 RVEs (mixed), 5 of 20 steps",
              synth.biaxial_shear_2d(macro=8, rve=32), 5, {}),
             ("c3-shaped 3D 4^3 Hex8 macro, 512 qps, 8/12/16^3 RVEs (mixed), 4 of 10 steps",
              synth.uniaxial_3d_uneven(macro=4), 4, {})]
    from paper_1908_08292_gb300 import FehmmError
    out = []
    for name, p, steps, opts in cases:
        row = {"case": name}
        for scheme in ("nested", "alternating"):
            recs, drv = [], None
            try:
                drv = LoadStepDriver(p, scheme=scheme, graphs=True, **opts)
                drv.load_step(1)  # warm-up: module load, graph capture (state then restarts)
                drv.close()
                drv = LoadStepDriver(p, scheme=scheme, graphs=True, **opts)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for k in range(1, steps + 1):
                    recs.append(drv.load_step(k))
                torch.cuda.synchronize()
                row[scheme] = {"seconds": time.perf_counter() - t0,
                               "macro_iters": int(sum(r["macro_iters"] for r in recs)),
                               "micro_newton_iters": int(sum(sum(r["micro_newton"]) for r in recs)),
                               "all_converged": bool(all(r["converged"] for r in recs)),
                               "macro_iters_per_step": [r["macro_iters"] for r in recs]}
                # where the RVE time goes: the same load path once more, instrumented (eager): RVE
                # kernel time and the PCG iterations of the Newton corrections vs the transfer
                drv.close()
                drv = LoadStepDriver(p, scheme=scheme, graphs=False, **opts)
                drv.rve_events, drv.iter_log = [], []
                for k in range(1, steps + 1):
                    drv.load_step(k)
                torch.cuda.synchronize()
                its = [t.cpu().numpy() for t in drv.iter_log]
                row[scheme]["rve_kernel_seconds"] = sum(a.elapsed_time(b) for a, b in drv.rve_events) / 1e3
                row[scheme]["rve_passes"] = len(its)
                row[scheme]["pcg_newton_per_rve"] = float(sum(i[:, 1].sum() for i in its) / p.n_qp)
                row[scheme]["pcg_transfer_per_rve"] = float(sum(i[:, 2].sum() for i in its) / p.n_qp)
            except FehmmError as e:  # a scheme that fails on a case is a result, not a crash
                row[scheme] = {"failed": str(e), "steps_done": len(recs)}
            finally:
                if drv is not None:
                    drv.close()
        if "seconds" in row["nested"] and "seconds" in row["alternating"]:
            row["speedup_alternating"] = row["nested"]["seconds"] / row["alternating"]["seconds"]
        out.append(row)
    print(json.dumps({"metric": "load-path wall time, nested (Algorithm 1) vs alternating (Algorithm 2)",
                      "workload": "schemes", "n_gpus": 1, "unit": "s", "higher_is_better": False, "cases": out}))


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
    ap.add_argument("--mode", default="path", choices=["path", "iteration"],
                    help="path: whole load steps 1/10/20 of the load path (default); iteration: macro iteration 1 "
                         "of --step-index from the zero state (short runs for profiling)")
    ap.add_argument("--precond", default="mg", choices=["mg", "jacobi"],
                    help="RVE PCG preconditioner: multigrid V-cycle (default; 2D) or block-Jacobi")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "schemes", "hconv", "mlp"],
                    help="c2: 2D 4096 RVEs of 32x32 (default, the headline); c3: 3D 4096 uneven Hex8 RVEs; "
                         "c4: surrogate training; c5: surrogate+fallback vs plain macro iteration; "
                         "schemes: nested vs alternating load paths; hconv: micro mesh convergence and the KUBC "
                         "modelling error")
    ap.add_argument("--c4-samples", type=int, default=204800)
    ap.add_argument("--c4-holdout", type=int, default=10240)
    ap.add_argument("--c4-epochs", type=int, default=2400)
    ap.add_argument("--c4-lr", type=float, default=1e-3, help="peak AdamW learning rate (cosine decay to 1/100)")
    ap.add_argument("--c4-out-scale", type=float, default=0.0,
                    help="scale of the network's initial output weights (0: zero output layer)")
    ap.add_argument("--c4-hessian-origin", type=int, default=1,
                    help="subtract the network's value, gradient and Hessian at E = 0 (1) or value and gradient (0)")
    ap.add_argument("--c4-save", default=None, help="write the trained surrogate to this file")
    ap.add_argument("--autotune", default="auto", choices=["auto", "on", "off"],
                    help="path mode: autotune the solver settings before the timed steps (auto: c3 only)")
    ap.add_argument("--c4-poly", type=int, default=6,
                    help="maximum degree (3-6) of the polynomial part fitted before the network; 0: none")
    ap.add_argument("--c4-load", default=None, help="c5: use the surrogate in this file instead of training one")
    ap.add_argument("--c5-radius", type=float, default=0.3)
    ap.add_argument("--mlp-points", type=int, default=32768, help="mlp: inference points per call")
    ap.add_argument("--c5-step", type=int, default=10)
    ap.add_argument("--c5-audit-stride", type=int, default=64)
    args = ap.parse_args()
    _SIZE["workload"] = args.workload
    _SIZE["precond"] = args.precond
    _SIZE["macro"] = args.macro if args.macro is not None else (MACRO_C3 if args.workload == "c3" else MACRO)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_c4(args)
    elif args.workload == "schemes":
        run_schemes(args)
    elif args.workload == "hconv":
        run_hconv(args)
    elif args.workload == "mlp":
        run_mlp(args)
    elif args.workload == "c5":
        _SIZE["macro"] = args.macro if args.macro is not None else 8
        args.macro = _SIZE["macro"]
        run_c5(args)
    elif args.mode == "iteration":
        run_gpu_iteration(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
