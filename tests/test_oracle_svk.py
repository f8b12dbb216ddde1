"""Pins of the St. Venant-Kirchhoff law (the paper's "linear elasticity with geometrical
nonlinearity", Sec. 6) and of the periodic RVE oracle run with it: P = dpsi/dF and A = dP/dF by
finite differences, the small-strain limit equals Hooke's tensor, objectivity, the RVE's literal
B^T CC B + G_hat tangent equals the assembled one, a homogeneous RVE reproduces the pointwise law,
and Pbar = dWbar/dFbar, Abar = dPbar/dFbar for a heterogeneous RVE."""
import numpy as np
import pytest

import synth
from oracle import material as mat
from oracle.rve import PeriodicRVE


@pytest.mark.parametrize("d", [2, 3])
def test_svk_derivatives_by_finite_differences(d):
    lam, mu = 1.3, 0.7
    F = synth.random_F(81, 1, d, 0.2)[0]
    P = mat.svk_P(F, lam, mu)
    A = mat.svk_A(F, lam, mu)
    h = 1e-6
    for k in range(d):
        for l in range(d):
            E = np.zeros((d, d))
            E[k, l] = h
            assert abs((mat.svk_psi(F + E, lam, mu) - mat.svk_psi(F - E, lam, mu)) / (2 * h) - P[k, l]) < 1e-8
            np.testing.assert_allclose((mat.svk_P(F + E, lam, mu) - mat.svk_P(F - E, lam, mu)) / (2 * h),
                                       A[:, :, k, l], atol=1e-7)


@pytest.mark.parametrize("d", [2, 3])
def test_svk_small_strain_limit_and_objectivity(d):
    lam, mu = 1.3, 0.7
    np.testing.assert_allclose(mat.svk_A(np.eye(d), lam, mu), mat.hooke(lam, mu, d), atol=1e-14)
    F = synth.random_F(82, 1, d, 0.2)[0]
    th = 0.4
    Q = np.eye(d)
    Q[:2, :2] = [[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]
    assert abs(mat.svk_psi(Q @ F, lam, mu) - mat.svk_psi(F, lam, mu)) < 1e-14
    np.testing.assert_allclose(mat.svk_P(Q @ F, lam, mu), Q @ mat.svk_P(F, lam, mu), atol=1e-13)


@pytest.mark.parametrize("d,n", [(2, 6), (3, 3)])
def test_svk_rve_literal_tangent_and_homogeneous_case(d, n):
    ph = (synth.uniform(83, np.arange(n ** d), 1)[:, 0] > 0.5).astype(np.uint8)
    rve = PeriodicRVE(n, d, ph, [1.0, 5.0], [0.3, 0.25], law="svk")
    F = synth.random_F(84, 1, d, 0.1)[0]
    w = 0.01 * synth.random_field(85, 1, rve.n_dof, 1.0)[0]
    w[:d] = 0.0
    assert abs(rve.tangent(w, F) - rve.tangent_literal(w, F)).max() < 1e-12
    hom = PeriodicRVE(n, d, np.zeros(n ** d, np.uint8), [2.0, 2.0], [0.3, 0.3], law="svk")
    out = hom.solve(F, rtol=1e-14)
    lam, mu = mat.lame(2.0, 0.3)
    np.testing.assert_allclose(out["P"], mat.svk_P(F, lam, mu), atol=1e-13)
    np.testing.assert_allclose(out["A"], mat.svk_A(F, lam, mu), atol=1e-12)


def test_svk_rve_energy_consistency():
    n = 6
    ph = synth.phase_from_inclusions(n, 2, [[0.45, 0.5]], [0.3])
    rve = PeriodicRVE(n, 2, ph, [1.0, 10.0], [0.3, 0.3], law="svk")
    F = np.array([[1.06, 0.04], [-0.02, 0.97]])
    out = rve.solve(F, rtol=1e-14)
    h = 1e-5
    for k in range(2):
        for l in range(2):
            E = np.zeros((2, 2))
            E[k, l] = h
            p, m = rve.solve(F + E, rtol=1e-14, tangent=False), rve.solve(F - E, rtol=1e-14, tangent=False)
            assert abs((p["W"] - m["W"]) / (2 * h) - out["P"][k, l]) < 1e-8
            np.testing.assert_allclose((p["P"] - m["P"]) / (2 * h), out["A"][:, :, k, l], atol=1e-7)
