"""Pins of the KUBC (Dirichlet-coupled) RVE oracle against facts fixed by the mathematics and the
paper: the homogeneous RVE is the pointwise law; Pbar = dWbar/dFbar and Abar = dPbar/dFbar (finite
differences); Hill-Mandel; Hill's ordering of small-strain effective tangents (Voigt >= KUBC >=
periodic >= Reuss); and the modelling error of Dirichlet coupling (Sec. 4, Eq. ModelingError)
shrinking as the sampling domain holds more cells."""
import numpy as np
import pytest

import synth
from oracle import material as mat
from oracle.kubc import DirichletRVE
from oracle.rve import PeriodicRVE


def mandel_energy(A, eps):
    return float(np.einsum("ij,ijkl,kl->", eps, A, eps))


def random_sym(seed, d, n):
    e = synth.random_field(seed, n, d * d, 1.0).reshape(n, d, d)
    return 0.5 * (e + e.transpose(0, 2, 1))


@pytest.mark.parametrize("d", [2, 3])
def test_homogeneous_kubc_rve_is_pointwise_law(d):
    n = 4
    rve = DirichletRVE(n, d, np.zeros(n ** d, np.uint8), [2.0, 2.0], [0.3, 0.3])
    F = synth.random_F(71, 1, d, 0.15)[0]
    out = rve.solve(F)
    lam, mu = mat.lame(2.0, 0.3)
    assert out["status"] == 0 and out["newton_iters"] == 0
    np.testing.assert_allclose(out["P"], mat.P_of_F(F, lam, mu), atol=1e-13)
    np.testing.assert_allclose(out["A"], mat.A_of_F(F, lam, mu), atol=1e-12)


def test_kubc_energy_consistency_and_hill_mandel():
    n = 6
    ph = synth.phase_from_inclusions(n, 2, [[0.45, 0.55]], [0.3])
    rve = DirichletRVE(n, 2, ph, [1.0, 10.0], [0.3, 0.3])
    F = np.array([[1.08, 0.05], [-0.02, 0.95]])
    out = rve.solve(F, rtol=1e-14)
    # Hill-Mandel: <P : F> = Pbar : Fbar at equilibrium, and <F> = Fbar (w = 0 on the boundary)
    Fq = rve.F_at_qps(out["w"], F)
    Pq = mat.P_of_F(Fq, rve.lam_e[:, None], rve.mu_e[:, None])
    assert abs(rve.wdet * np.einsum("eqiJ,eqiJ->", Pq, Fq) - np.sum(out["P"] * F)) < 1e-12
    np.testing.assert_allclose(out["F_mean"], F, atol=1e-14)
    h = 1e-5
    for k in range(2):
        for l in range(2):
            E = np.zeros((2, 2))
            E[k, l] = h
            Wp, Wm = rve.solve(F + E, rtol=1e-14, tangent=False), rve.solve(F - E, rtol=1e-14, tangent=False)
            assert abs((Wp["W"] - Wm["W"]) / (2 * h) - out["P"][k, l]) < 1e-8
            np.testing.assert_allclose((Wp["P"] - Wm["P"]) / (2 * h), out["A"][:, :, k, l], atol=1e-7)


@pytest.mark.parametrize("d", [2, 3])
def test_hill_ordering_voigt_kubc_periodic_reuss(d):
    n = 8 if d == 2 else 4
    if d == 2:
        ph = synth.phase_from_inclusions(n, 2, [[0.4, 0.55]], [0.3])
    else:
        ph = synth.sphere_rve(n, 1, 0.2, [[0.45, 0.5, 0.55]])
    E, nu = [1.0, 10.0], [0.3, 0.3]
    I = np.eye(d)
    Ak = DirichletRVE(n, d, ph, E, nu).solve(I)["A"]
    Ap = PeriodicRVE(n, d, ph, E, nu).solve(I, rtol=1e-14)["A"]
    lam, mu = mat.lame(np.array(E), np.array(nu))
    phi = np.array([1 - ph.mean(), ph.mean()])
    CV = sum(phi[i] * mat.A_of_F(I, lam[i], mu[i]) for i in range(2))
    for eps in random_sym(73, d, 6):
        ev, ek, ep = mandel_energy(CV, eps), mandel_energy(Ak, eps), mandel_energy(Ap, eps)
        assert ev >= ek - 1e-12 and ek >= ep - 1e-12, (ev, ek, ep)
        # Reuss: both phases have nu = 0.3, so C_i = E_i C_1 and the Reuss energy is the harmonic
        # mean of the phase energies
        cr = 1.0 / sum(phi[i] / mandel_energy(mat.A_of_F(I, lam[i], mu[i]), eps) for i in range(2))
        assert ep >= cr - 1e-12


def test_kubc_modelling_error_decreases_with_more_cells():
    """k x k tilings of one periodic cell: the KUBC tangent stiffens the response less and less
    (boundary layer of relative width ~1/k) and stays above the periodic one."""
    m = 4
    cell = synth.phase_from_inclusions(m, 2, [[0.5, 0.5]], [0.3]).reshape(m, m)
    E, nu = [1.0, 10.0], [0.3, 0.3]
    I = np.eye(2)
    Ap = PeriodicRVE(m, 2, cell.reshape(-1), E, nu).solve(I, rtol=1e-14)["A"]
    eps = np.array([[0.6, 0.3], [0.3, -0.2]])
    e_per = mandel_energy(Ap, eps)
    gaps = []
    for k in (1, 2, 3):
        ph = np.tile(cell, (k, k)).reshape(-1)
        Ak = DirichletRVE(m * k, 2, ph, E, nu).solve(I)["A"]
        gaps.append(mandel_energy(Ak, eps) - e_per)
    assert all(g > 0 for g in gaps)
    assert gaps[0] > gaps[1] > gaps[2]
