"""Parity of the CUDA 3D (Hex8) RVE batch with the FP64 oracle.

Tolerances as in 2D (relative Frobenius norm per quadrature point, P floored at 1e-3 x the matrix
Young's modulus): FP64 mode 1e-10 on P and A, mixed mode 1e-5."""
import numpy as np
import pytest

import synth
from oracle import material as mat
from oracle.rve import PeriodicRVE
from gpu_harness import gpu_batch, rel_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
STRICT = dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-9, cond_rtol=1e-11)


def check(out, refs, tol):
    for q, ref in enumerate(refs):
        assert out["status"][q] == 0, (q, out["status"][q])
        eP = rel_err(out["P"][q], ref["P"], 1e-3)
        eA = rel_err(out["A"][q], ref["A"], 1e-3)
        assert eP < tol and eA < tol, (q, eP, eA)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_small_sizes_one_launch(precision):
    """n = 2 (the 27-point neighbourhood wraps onto itself), 3 (odd), 4 and 6 in one launch."""
    sizes = [2, 3, 4, 6]
    u = synth.uniform(601, np.arange(len(sizes)), 4)
    phases, E, nu = [], [], []
    for k, n in enumerate(sizes):
        phases.append(synth.phase_from_inclusions(n, 3, [u[k, :3]], [0.2 + 0.15 * u[k, 3]]))
        E.append([1.0, 10.0])
        nu.append([0.3, 0.25])
    qp_rve = np.array([3, 0, 1, 2, 3, 2])
    Fs = synth.random_F(602, len(qp_rve), 3, 0.08)
    opts = STRICT if precision == "fp64" else {}
    out = gpu_batch(3, precision, sizes, phases, E, nu, qp_rve, Fs, **opts)
    refs = [PeriodicRVE(sizes[r], 3, phases[r], E[r], nu[r]).solve(F, rtol=1e-14, atol=1e-16)
            for r, F in zip(qp_rve, Fs)]
    check(out, refs, TOL[precision])
    for q, r in enumerate(qp_rve):
        assert np.abs(out["w"][q] - refs[q]["w"]).max() < (1e-10 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_workload_3d_generator_rves(precision):
    """8^3 RVEs of the 3D workload generator (1-4 spheres, ratio 10) along its uniaxial load path."""
    p = synth.uniaxial_3d_uneven(macro=1, sizes=(8,), n_rve=3)
    Fs = np.array([np.diag([1.0 + s, 1.0 - 0.3 * s, 1.0 - 0.3 * s]) for s in (0.02, 0.1, 0.2)])
    opts = STRICT if precision == "fp64" else {}
    out = gpu_batch(3, precision, p.rve_n, p.rve_phase, p.rve_E, p.rve_nu, np.arange(3), Fs, flags=4, **opts)
    refs = [PeriodicRVE(8, 3, p.rve_phase[r], p.rve_E[r], p.rve_nu[r]).solve(Fs[r], rtol=1e-14, atol=1e-16)
            for r in range(3)]
    check(out, refs, TOL[precision])
    for q in range(3):  # homogenised energy <psi>
        assert abs(out["W"][q] - refs[q]["W"]) <= TOL[precision] * abs(refs[q]["W"])


_REF16 = {}


def _ref16():
    """One 16^3 RVE of the 3D workload generator (the largest grid of that workload: 12288 dofs,
    three coarse levels 8, 4, 2) at a tension-shear Fbar, solved once by the oracle (about 100 s
    of sparse LU) and shared by the two precisions."""
    if not _REF16:
        p = synth.uniaxial_3d_uneven(macro=1, sizes=(16,), n_rve=1)
        F = np.eye(3) + np.array([[0.08, 0.04, 0.0], [0.02, -0.02, 0.03], [0.0, 0.01, -0.02]])
        ref = PeriodicRVE(16, 3, p.rve_phase[0], p.rve_E[0], p.rve_nu[0]).solve(F, rtol=1e-13, atol=1e-16)
        _REF16.update(p=p, F=F, ref=ref)
    return _REF16


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_workload_3d_16cubed_rve(precision):
    """The 16^3 Hex8 RVE of the 3D workload (largest scratch and multigrid depth) against
    the oracle: P and A per point at 1e-10 (FP64) / 1e-5 (mixed), with the 8^3 and 12^3 grids of
    the same workload in the same launch."""
    r16 = _ref16()
    p = r16["p"]
    small = synth.uniaxial_3d_uneven(macro=1, sizes=(8, 12), n_rve=2, seed=1013)
    sizes = [16] + [int(n) for n in small.rve_n]
    phases = [p.rve_phase[0]] + list(small.rve_phase)
    E = [p.rve_E[0]] + list(small.rve_E)
    nu = [p.rve_nu[0]] + list(small.rve_nu)
    Fs = np.stack([r16["F"], r16["F"], r16["F"]])
    opts = STRICT if precision == "fp64" else {}
    out = gpu_batch(3, precision, sizes, phases, E, nu, np.arange(3), Fs, **opts)
    refs = [r16["ref"]] + [PeriodicRVE(sizes[k], 3, phases[k], E[k], nu[k]).solve(Fs[k], rtol=1e-14, atol=1e-16)
                           for k in (1, 2)]
    check(out, refs, TOL[precision])
    assert np.abs(out["w"][0] - r16["ref"]["w"]).max() < (1e-10 if precision == "fp64" else 1e-6)


def test_homogeneous_rve_is_pointwise_law_3d():
    n = 4
    Fs = synth.random_F(603, 2, 3, 0.1)
    out = gpu_batch(3, "fp64", [n], [np.zeros(n ** 3, np.uint8)], [[2.0, 2.0]], [[0.3, 0.3]], [0, 0], Fs, **STRICT)
    lam, mu = mat.lame(2.0, 0.3)
    for q in range(2):
        assert out["status"][q] == 0 and out["iters"][q][0] == 0
        np.testing.assert_allclose(out["P"][q], mat.P_of_F(Fs[q], lam, mu), atol=1e-13)
        np.testing.assert_allclose(out["A"][q], mat.A_of_F(Fs[q], lam, mu), atol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_failed_start_retried_by_load_continuation(precision):
    """A start fluctuation that folds elements (J <= 0 before the first Newton step) fails with
    retry_stages = 0 and, with retry_stages = 4, is re-solved from zero by load continuation to
    the oracle's continuation result (which equals the direct solve from zero)."""
    n = 4
    phase = synth.phase_from_inclusions(n, 3, [[0.45, 0.5, 0.55]], [0.3])
    E, nu = [1.0, 10.0], [0.3, 0.25]
    F = synth.random_F(611, 1, 3, 0.2)
    w_bad = np.zeros(3 * n ** 3)
    w_bad[3] = 0.8  # x-displacement of node 1: dw_x/dX_1 about -3 in the next elements
    rve = PeriodicRVE(n, 3, phase, E, nu)
    assert rve.newton(F[0], w_bad)[1] == 2  # the start state is inadmissible (J <= 0)
    opts = dict(STRICT) if precision == "fp64" else {}
    off = gpu_batch(3, precision, [n], [phase], [E], [nu], [0], F, w0=[w_bad], retry_stages=0, **opts)
    assert off["status"][0] == 2
    on = gpu_batch(3, precision, [n], [phase], [E], [nu], [0], F, w0=[w_bad], retry_stages=4, **opts)
    ref = rve.solve(F[0], rtol=1e-14, atol=1e-16, stages=4)
    check(on, [ref], TOL[precision])
    assert on["iters"][0][0] > 4  # Newton iterations summed over the first try and the four increments


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multigrid_and_block_jacobi_agree_3d(precision):
    """3D: both preconditioners reach the oracle's P and A; the multigrid V-cycle (n = 8: coarse
    levels 4, 2; n = 12: 6, 3) needs far fewer PCG iterations; n = 10 has no hierarchy."""
    sizes = [8, 12, 10]
    u = synth.uniform(641, np.arange(len(sizes)), 5)
    phases = [synth.sphere_rve(n, 1, 0.15 + 0.1 * u[k, 3], [u[k, :3]]) for k, n in enumerate(sizes)]
    E = [[1.0, 10.0]] * len(sizes)
    nu = [[0.3, 0.3]] * len(sizes)
    Fs = synth.random_F(642, len(sizes), 3, 0.08)
    opts = STRICT if precision == "fp64" else {}
    mg = gpu_batch(3, precision, sizes, phases, E, nu, np.arange(len(sizes)), Fs, precond=1, **opts)
    bj = gpu_batch(3, precision, sizes, phases, E, nu, np.arange(len(sizes)), Fs, precond=0, **opts)
    refs = [PeriodicRVE(n, 3, phases[k], E[k], nu[k]).solve(Fs[k], rtol=1e-14, atol=1e-16)
            for k, n in enumerate(sizes)]
    check(mg, refs, TOL[precision])
    check(bj, refs, TOL[precision])
    for q in (0, 1):
        assert mg["iters"][q][1] < 0.3 * bj["iters"][q][1], (sizes[q], mg["iters"][q], bj["iters"][q])
        assert mg["iters"][q][2] < 0.3 * bj["iters"][q][2], (sizes[q], mg["iters"][q], bj["iters"][q])
    # n = 10 runs block-Jacobi either way; the 3D apply sums with float atomics, so iteration
    # counts may differ by the order of the sums
    assert abs(int(mg["iters"][2][1]) - int(bj["iters"][2][1])) <= max(2, 0.02 * bj["iters"][2][1])
