"""Pins of the oracle's neo-Hookean law (paper Sec. 6) against values and identities that do not
come from the oracle itself: the paper's printed Lame table, finite differences of the free energy,
the small-strain (Hooke) limit, objectivity and a uniaxial closed form."""
import os

import numpy as np
import pytest

import synth
from oracle import material as mat

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_lame_table_matches_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lame_table.txt")) if l.strip() and not l.startswith("#")]
    for _, E, nu, lam_p, mu_p in rows:
        lam, mu = mat.lame(float(E), float(nu))
        assert abs(lam - float(lam_p)) <= 0.006
        assert abs(mu - float(mu_p)) <= 0.006


@pytest.mark.parametrize("d", [2, 3])
def test_P_is_derivative_of_psi(d):
    lam, mu = mat.lame(np.array([1.0, 10.0]), np.array([0.3, 0.3]))
    F = synth.random_F(11, 2, d, 0.2)
    h = 1e-6
    P = mat.P_of_F(F, lam, mu)
    for i in range(d):
        for j in range(d):
            E = np.zeros((d, d))
            E[i, j] = h
            fd = (mat.psi(F + E, lam, mu) - mat.psi(F - E, lam, mu)) / (2 * h)
            np.testing.assert_allclose(P[:, i, j], fd, rtol=0, atol=2e-9 * np.abs(P).max())


@pytest.mark.parametrize("d", [2, 3])
def test_A_is_derivative_of_P(d):
    lam, mu = mat.lame(np.array([1.0, 10.0]), np.array([0.3, 0.3]))
    F = synth.random_F(12, 2, d, 0.2)
    h = 1e-6
    A = mat.A_of_F(F, lam, mu)
    for k in range(d):
        for l in range(d):
            E = np.zeros((d, d))
            E[k, l] = h
            fd = (mat.P_of_F(F + E, lam, mu) - mat.P_of_F(F - E, lam, mu)) / (2 * h)
            np.testing.assert_allclose(A[..., k, l], fd, rtol=0, atol=2e-8 * np.abs(A).max())


@pytest.mark.parametrize("d", [2, 3])
def test_CC_is_twice_derivative_of_S(d):
    lam, mu = mat.lame(4.0, 0.25)
    F = synth.random_F(13, 1, d, 0.2)[0]
    C = F.T @ F
    h = 1e-6
    CC = mat.CC_of_C(C, lam, mu)
    for k in range(d):
        for l in range(d):
            E = np.zeros((d, d))
            E[k, l] += h / 2
            E[l, k] += h / 2
            fd = 2 * (mat.S_of_C(C + E, lam, mu) - mat.S_of_C(C - E, lam, mu)) / (2 * h)
            np.testing.assert_allclose(CC[:, :, k, l], fd, atol=1e-7 * np.abs(CC).max())


@pytest.mark.parametrize("d", [2, 3])
def test_small_strain_limit_is_hooke(d):
    lam, mu = mat.lame(7.0, 0.3)
    np.testing.assert_allclose(mat.CC_of_C(np.eye(d), lam, mu), mat.hooke(lam, mu, d), atol=1e-13)
    np.testing.assert_allclose(mat.A_of_F(np.eye(d), lam, mu), mat.hooke(lam, mu, d), atol=1e-13)
    assert abs(mat.psi(np.eye(d), lam, mu)) < 1e-15
    np.testing.assert_allclose(mat.P_of_F(np.eye(d), lam, mu), 0, atol=1e-15)


def test_stress_free_reference_and_objectivity():
    lam, mu = mat.lame(2.0, 0.3)
    F = synth.random_F(14, 4, 3, 0.2)
    # rotation from a skew matrix via Cayley
    Wk = np.array([[0, -0.3, 0.2], [0.3, 0, -0.5], [-0.2, 0.5, 0]])
    Q = np.linalg.solve(np.eye(3) - Wk, np.eye(3) + Wk)
    np.testing.assert_allclose(mat.psi(Q @ F, lam, mu), mat.psi(F, lam, mu), rtol=1e-13)
    np.testing.assert_allclose(mat.P_of_F(Q @ F, lam, mu), Q @ mat.P_of_F(F, lam, mu), atol=1e-13)


def test_uniaxial_plane_strain_closed_form():
    """F = diag(s, t) with P_22 = 0: S_22 = lam/2 (s^2 t^2 - 1)/t^2 + mu (1 - 1/t^2) = 0
    gives t^2 = (lam/2 + mu)/(lam s^2/2 + mu) and P_11 = s [lam/2 (s^2 t^2 - 1)/s^2 + mu (1 - 1/s^2)]."""
    lam, mu = mat.lame(1.0, 0.3)
    s = 1.1
    t = np.sqrt((lam / 2 + mu) / (lam * s * s / 2 + mu))
    P = mat.P_of_F(np.diag([s, t]), lam, mu)
    assert abs(P[1, 1]) < 1e-15
    P11 = s * (lam / 2 * (s * s * t * t - 1) / (s * s) + mu * (1 - 1 / (s * s)))
    assert abs(P[0, 0] - P11) < 1e-15
