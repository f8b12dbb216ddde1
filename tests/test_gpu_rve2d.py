"""Parity of the CUDA 2D RVE batch (C-ABI fehmm_rve_solve) with the FP64 oracle.

Tolerances (relative Frobenius norm per quadrature point; the P norm is floored at
1e-3 x the matrix Young's modulus): FP64 mode 1e-10 on P and A; mixed mode 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle.rve import PeriodicRVE
from gpu_harness import gpu_batch, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
STRICT = dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-8, cond_rtol=1e-11)


def oracle_solve(n, phase, E, nu, Fb, w0=None):
    return PeriodicRVE(n, 2, phase, E, nu).solve(Fb, w0, rtol=1e-14, atol=1e-16)


def check(out, refs, tol, check_W=False):
    for q, ref in enumerate(refs):
        assert out["status"][q] == 0, (q, out["status"][q])
        assert rel_err(out["P"][q], ref["P"], 1e-3) < tol, (q, rel_err(out["P"][q], ref["P"], 1e-3))
        assert rel_err(out["A"][q], ref["A"], 1e-3) < tol, (q, rel_err(out["A"][q], ref["A"], 1e-3))
        if check_W:
            assert abs(out["W"][q] - ref["W"]) <= tol * max(abs(ref["W"]), 1e-3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_rve_random_F(precision):
    n = 8
    phase = synth.phase_from_inclusions(n, 2, [[0.5, 0.5]], [0.25])
    Fs = synth.random_F(101, 12, 2, 0.15)
    opts = STRICT if precision == "fp64" else dict(newton_rtol=1e-12, newton_atol=1e-15)
    out = gpu_batch(2, precision, [n], [phase], [[1.0, 10.0]], [[0.3, 0.3]], np.zeros(12), Fs,
                    flags=4, **opts)
    refs = [oracle_solve(n, phase, [1.0, 10.0], [0.3, 0.3], F) for F in Fs]
    check(out, refs, TOL[precision], check_W=True)
    for q, ref in enumerate(refs):
        assert np.abs(out["w"][q] - ref["w"]).max() < (1e-10 if precision == "fp64" else 1e-7)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_sizes_one_launch(precision):
    """n = 2 (degenerate: the 9-point stencil wraps onto itself), 4, 6, 16 and 32 in one batch,
    several phases, random stiffness contrast; ragged and repeated microstructures."""
    sizes = [2, 4, 6, 16, 32]
    u = synth.uniform(202, np.arange(len(sizes)), 4)
    phases, E, nu = [], [], []
    for k, n in enumerate(sizes):
        ph = synth.phase_from_inclusions(n, 2, [u[k, :2]], [0.15 + 0.2 * u[k, 2]])
        if n >= 4:
            ph[: n] = 2  # a third phase along the first row
        phases.append(ph)
        E.append([1.0, 5.0 + 40.0 * u[k, 3], 3.0])
        nu.append([0.3, 0.25, 0.2])
    qp_rve = np.array([0, 1, 2, 3, 4, 4, 3, 1])
    Fs = synth.random_F(203, len(qp_rve), 2, 0.12)
    opts = STRICT if precision == "fp64" else {}
    out = gpu_batch(2, precision, sizes, phases, E, nu, qp_rve, Fs, **opts)
    refs = [PeriodicRVE(sizes[r], 2, phases[r], E[r], nu[r]).solve(F, rtol=1e-14, atol=1e-16)
            for r, F in zip(qp_rve, Fs)]
    check(out, refs, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_workload_2d_sized_rves(precision):
    """32x32 RVEs drawn from the 2D workload generator (the benchmark's RVEs) at
    deformation gradients along its load path (biaxial 30% + shear 0.3)."""
    p = synth.biaxial_shear_2d(macro=1, rve=32, n_rve=4)
    F_end = p.extra["F_end"]
    lams = [0.05, 0.3, 0.7, 1.0]
    Fs = np.array([np.eye(2) + l * (F_end - np.eye(2)) for l in lams])
    opts = STRICT if precision == "fp64" else {}
    out = gpu_batch(2, precision, p.rve_n, p.rve_phase, p.rve_E, p.rve_nu, np.arange(4), Fs, **opts)
    refs = [PeriodicRVE(32, 2, p.rve_phase[r], p.rve_E[r], p.rve_nu[r]).solve(Fs[r], rtol=1e-14, atol=1e-16)
            for r in range(4)]
    check(out, refs, TOL[precision])


def test_homogeneous_and_identity_cases():
    """Homogeneous RVE: w stays 0 and P, A equal the pointwise law; F = I gives P = 0."""
    from oracle import material as mat
    n = 8
    Fs = np.array([[[1.2, 0.1], [-0.05, 0.9]], np.eye(2)])
    out = gpu_batch(2, "fp64", [n], [np.zeros(n * n, np.uint8)], [[2.0, 2.0]], [[0.3, 0.3]], [0, 0], Fs, **STRICT)
    lam, mu = mat.lame(2.0, 0.3)
    for q in range(2):
        assert out["status"][q] == 0
        np.testing.assert_allclose(out["P"][q], mat.P_of_F(Fs[q], lam, mu), atol=1e-13)
        np.testing.assert_allclose(out["A"][q], mat.A_of_F(Fs[q], lam, mu), atol=1e-12)
        assert np.abs(out["w"][q]).max() < 1e-13
        assert out["iters"][q][0] == 0  # R_0 = 0: no Newton step taken


def test_negative_jacobian_reported():
    n = 8
    phase = synth.phase_from_inclusions(n, 2, [[0.5, 0.5]], [0.25])
    Fs = np.array([[[1.0, 0.0], [0.0, -0.5]], [[1.05, 0.0], [0.0, 1.0]]])
    out = gpu_batch(2, "mixed", [n], [phase], [[1.0, 10.0]], [[0.3, 0.3]], [0, 0], Fs)
    assert out["status"][0] == 2
    assert out["status"][1] == 0


def test_warm_start_and_alternating_single_iteration():
    """A warm start from the converged fluctuation needs no Newton step; max_newton = 1 (one
    micro iteration, Algorithm 2) returns the oracle's single-step state."""
    n = 8
    phase = synth.phase_from_inclusions(n, 2, [[0.45, 0.5]], [0.3])
    Fb = np.array([[1.1, 0.05], [0.0, 0.95]])
    rve = PeriodicRVE(n, 2, phase, [1.0, 10.0], [0.3, 0.3])
    ref = rve.solve(Fb, rtol=1e-14)
    out = gpu_batch(2, "fp64", [n], [phase], [[1.0, 10.0]], [[0.3, 0.3]], [0], Fb[None], w0=[ref["w"]],
                    newton_rtol=1e-8, newton_atol=1e-13)
    assert out["iters"][0][0] == 0 and out["status"][0] == 0
    assert rel_err(out["P"][0], ref["P"], 1e-3) < 1e-12
    one = rve.solve(Fb, rtol=1e-14, max_steps=1)
    out1 = gpu_batch(2, "fp64", [n], [phase], [[1.0, 10.0]], [[0.3, 0.3]], [0], Fb[None], max_newton=1,
                     cg_rtol=1e-13, cond_rtol=1e-12)
    assert out1["iters"][0][0] == 1 and out1["status"][0] == 1  # cap after one step
    assert np.abs(out1["w"][0] - one["w"]).max() < 1e-11
    assert rel_err(out1["P"][0], one["P"], 1e-3) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_failed_start_retried_by_load_continuation(precision):
    """A start fluctuation that folds elements (J <= 0 before the first Newton step) fails with
    retry_stages = 0 and, with retry_stages = 4, is re-solved from zero by load continuation to
    the oracle's continuation result."""
    n = 8
    phase = synth.phase_from_inclusions(n, 2, [[0.4, 0.55]], [0.3])
    E, nu = [1.0, 10.0], [0.3, 0.3]
    F = synth.random_F(121, 1, 2, 0.2)
    w_bad = np.zeros(2 * n * n)
    w_bad[2] = 0.8  # x-displacement of node 1: dw_x/dX_1 about -6 in the next elements
    rve = PeriodicRVE(n, 2, phase, E, nu)
    assert rve.newton(F[0], w_bad)[1] == 2  # the start state is inadmissible (J <= 0)
    opts = dict(STRICT) if precision == "fp64" else dict(newton_rtol=1e-12, newton_atol=1e-15)
    off = gpu_batch(2, precision, [n], [phase], [E], [nu], [0], F, w0=[w_bad], retry_stages=0, **opts)
    assert off["status"][0] == 2
    on = gpu_batch(2, precision, [n], [phase], [E], [nu], [0], F, w0=[w_bad], retry_stages=4, **opts)
    ref = rve.solve(F[0], rtol=1e-14, atol=1e-16, stages=4)
    check(on, [ref], TOL[precision])
    assert on["iters"][0][0] > 4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multigrid_and_block_jacobi_agree(precision):
    """Both RVE preconditioners reach the oracle's P and A; the multigrid V-cycle needs far fewer
    PCG iterations (n = 24: coarse levels 12, 6, 3; n = 32: 16, 8, 4), and n = 10 (no hierarchy)
    falls back to block-Jacobi under either setting."""
    sizes = [24, 32, 10]
    u = synth.uniform(231, np.arange(len(sizes)), 4)
    phases, E, nu = [], [], []
    for k, n in enumerate(sizes):
        phases.append(synth.phase_from_inclusions(n, 2, [u[k, :2]], [0.2 + 0.1 * u[k, 2]]))
        E.append([1.0, 50.0])
        nu.append([0.3, 0.3])
    qp_rve = np.arange(len(sizes))
    Fs = synth.random_F(232, len(sizes), 2, 0.1)
    opts = STRICT if precision == "fp64" else dict(newton_rtol=1e-12, newton_atol=1e-15)
    mg = gpu_batch(2, precision, sizes, phases, E, nu, qp_rve, Fs, precond=1, **opts)
    bj = gpu_batch(2, precision, sizes, phases, E, nu, qp_rve, Fs, precond=0, **opts)
    refs = [PeriodicRVE(sizes[r], 2, phases[r], E[r], nu[r]).solve(F, rtol=1e-14, atol=1e-16)
            for r, F in zip(qp_rve, Fs)]
    check(mg, refs, TOL[precision])
    check(bj, refs, TOL[precision])
    for q in (0, 1):
        assert mg["iters"][q][1] < 0.3 * bj["iters"][q][1], (sizes[q], mg["iters"][q], bj["iters"][q])
        assert mg["iters"][q][2] < 0.3 * bj["iters"][q][2], (sizes[q], mg["iters"][q], bj["iters"][q])
    assert mg["iters"][2][1] == bj["iters"][2][1]
