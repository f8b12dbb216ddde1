"""Parity of the CUDA RVE batches with the FP64 oracle for the two further couplings and laws of
the paper's comparison: kinematically uniform boundary conditions (KUBC, Sec. 3.2; the oracle's
DirichletRVE on the (n+1)^d node lattice) and the St. Venant-Kirchhoff law (Sec. 6; the oracle's
PeriodicRVE with law="svk"), 2D and 3D, FP64 (1e-10) and mixed (1e-5) precision, multigrid and
block-Jacobi preconditioning."""
import numpy as np
import pytest

import synth
from gpu_harness import gpu_batch, rel_err
from oracle import material as mat
from oracle.kubc import DirichletRVE
from oracle.rve import PeriodicRVE

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
STRICT = {2: dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-8, cond_rtol=1e-11),
          3: dict(newton_rtol=1e-13, newton_atol=1e-15, cg_rtol=1e-9, cond_rtol=1e-11)}


def check(out, refs, tol, check_W=False):
    for q, ref in enumerate(refs):
        assert out["status"][q] == 0, (q, out["status"][q])
        eP, eA = rel_err(out["P"][q], ref["P"], 1e-3), rel_err(out["A"][q], ref["A"], 1e-3)
        assert eP < tol and eA < tol, (q, eP, eA)
        if check_W:
            assert abs(out["W"][q] - ref["W"]) <= tol * max(abs(ref["W"]), 1e-3)


def kubc_w_on_periodic_lattice(w, n, d):
    """The oracle's (n+1)^d-node fluctuation restricted to the n^d lattice of the kernels (node i
    of each axis for i < n; the planes x_c = 1 coincide with x_c = 0, where both are zero)."""
    w = np.asarray(w).reshape((n + 1,) * d + (d,))
    return w[(slice(0, n),) * d].reshape(-1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("precond", [1, 0])
def test_kubc_2d(precision, precond):
    """n = 2 (one free node), 6 and 8 (multigrid with pinned coarse boundary lines), 12, 32."""
    sizes = [2, 6, 8, 12, 32]
    u = synth.uniform(701, np.arange(len(sizes)), 4)
    phases = [synth.phase_from_inclusions(n, 2, [u[k, :2]], [0.15 + 0.2 * u[k, 2]]) for k, n in enumerate(sizes)]
    E = [[1.0, 5.0 + 40.0 * u[k, 3]] for k in range(len(sizes))]
    nu = [[0.3, 0.3]] * len(sizes)
    qp_rve = np.array([0, 1, 2, 3, 4, 4])
    Fs = synth.random_F(702, len(qp_rve), 2, 0.12)
    opts = dict(STRICT[2]) if precision == "fp64" else {}
    out = gpu_batch(2, precision, sizes, phases, E, nu, qp_rve, Fs, flags=4, bc=1, precond=precond, **opts)
    refs = [DirichletRVE(sizes[r], 2, phases[r], E[r], nu[r]).solve(F, rtol=1e-14, atol=1e-16)
            for r, F in zip(qp_rve, Fs)]
    check(out, refs, TOL[precision], check_W=True)
    for q, r in enumerate(qp_rve):
        wref = kubc_w_on_periodic_lattice(refs[q]["w"], sizes[r], 2)
        assert np.abs(out["w"][q] - wref).max() < (1e-10 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kubc_3d(precision):
    """Hex8 KUBC: n = 3, 4 (multigrid down to 2 nodes per axis), 6, 8 in one launch."""
    sizes = [3, 4, 6, 8]
    u = synth.uniform(711, np.arange(len(sizes)), 4)
    phases = [synth.phase_from_inclusions(n, 3, [u[k, :3]], [0.2 + 0.15 * u[k, 3]]) for k, n in enumerate(sizes)]
    E = [[1.0, 10.0]] * len(sizes)
    nu = [[0.3, 0.25]] * len(sizes)
    qp_rve = np.array([0, 1, 2, 3, 3])
    Fs = synth.random_F(712, len(qp_rve), 3, 0.08)
    opts = dict(STRICT[3]) if precision == "fp64" else {}
    out = gpu_batch(3, precision, sizes, phases, E, nu, qp_rve, Fs, flags=4, bc=1, **opts)
    refs = [DirichletRVE(sizes[r], 3, phases[r], E[r], nu[r]).solve(F, rtol=1e-14, atol=1e-16)
            for r, F in zip(qp_rve, Fs)]
    check(out, refs, TOL[precision], check_W=True)
    for q, r in enumerate(qp_rve):
        wref = kubc_w_on_periodic_lattice(refs[q]["w"], sizes[r], 3)
        assert np.abs(out["w"][q] - wref).max() < (1e-10 if precision == "fp64" else 1e-6)


def test_kubc_stiffer_than_periodic_at_small_strain():
    """Hill's ordering on the GPU: at small strain the KUBC tangent dominates the periodic one
    (e : A_KUBC : e >= e : A_per : e for random symmetric e) on the same microstructure."""
    n = 16
    phase = synth.phase_from_inclusions(n, 2, [[0.3, 0.6]], [0.3])
    F = np.eye(2)[None]  # the small-strain limit: w = 0, A is the effective elasticity tensor
    per = gpu_batch(2, "fp64", [n], [phase], [[1.0, 20.0]], [[0.3, 0.3]], [0], F, **STRICT[2])
    kub = gpu_batch(2, "fp64", [n], [phase], [[1.0, 20.0]], [[0.3, 0.3]], [0], F, bc=1, **STRICT[2])
    rng = np.random.default_rng(3)
    for _ in range(20):
        e = rng.standard_normal((2, 2))
        e = e + e.T
        a_p = np.einsum("ij,ijkl,kl", e, per["A"][0], e)
        a_k = np.einsum("ij,ijkl,kl", e, kub["A"][0], e)
        assert a_k >= a_p * (1 - 1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("precond", [1, 0])
def test_svk_2d(precision, precond):
    sizes = [2, 8, 16, 32]
    u = synth.uniform(731, np.arange(len(sizes)), 4)
    phases = [synth.phase_from_inclusions(n, 2, [u[k, :2]], [0.15 + 0.2 * u[k, 2]]) for k, n in enumerate(sizes)]
    E = [[1.0, 5.0 + 20.0 * u[k, 3]] for k in range(len(sizes))]
    nu = [[0.3, 0.3]] * len(sizes)
    qp_rve = np.array([0, 1, 2, 3, 3])
    Fs = synth.random_F(732, len(qp_rve), 2, 0.1)
    opts = dict(STRICT[2]) if precision == "fp64" else {}
    out = gpu_batch(2, precision, sizes, phases, E, nu, qp_rve, Fs, flags=4, law=1, precond=precond, **opts)
    refs = [PeriodicRVE(sizes[r], 2, phases[r], E[r], nu[r], law="svk").solve(F, rtol=1e-14, atol=1e-16)
            for r, F in zip(qp_rve, Fs)]
    check(out, refs, TOL[precision], check_W=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_svk_3d(precision):
    sizes = [3, 4, 8]
    u = synth.uniform(741, np.arange(len(sizes)), 4)
    phases = [synth.phase_from_inclusions(n, 3, [u[k, :3]], [0.2 + 0.15 * u[k, 3]]) for k, n in enumerate(sizes)]
    E = [[1.0, 10.0]] * len(sizes)
    nu = [[0.3, 0.25]] * len(sizes)
    qp_rve = np.array([0, 1, 2, 2])
    Fs = synth.random_F(742, len(qp_rve), 3, 0.08)
    opts = dict(STRICT[3]) if precision == "fp64" else {}
    out = gpu_batch(3, precision, sizes, phases, E, nu, qp_rve, Fs, flags=4, law=1, **opts)
    refs = [PeriodicRVE(sizes[r], 3, phases[r], E[r], nu[r], law="svk").solve(F, rtol=1e-14, atol=1e-16)
            for r, F in zip(qp_rve, Fs)]
    check(out, refs, TOL[precision], check_W=True)


@pytest.mark.parametrize("dim", [2, 3])
def test_svk_homogeneous_rve_is_pointwise_law(dim):
    n = 4
    Fs = synth.random_F(751, 2, dim, 0.1)
    out = gpu_batch(dim, "fp64", [n], [np.zeros(n ** dim, np.uint8)], [[2.0, 2.0]], [[0.3, 0.3]], [0, 0], Fs,
                    law=1, **STRICT[dim])
    lam, mu = mat.lame(2.0, 0.3)
    for q in range(2):
        assert out["status"][q] == 0 and out["iters"][q][0] == 0
        np.testing.assert_allclose(out["P"][q], mat.svk_P(Fs[q], lam, mu), atol=1e-13)
        np.testing.assert_allclose(out["A"][q], mat.svk_A(Fs[q], lam, mu), atol=1e-12)
