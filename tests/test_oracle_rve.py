"""Pins of the oracle's periodic RVE solver against facts fixed by the mathematics and the paper:
energy gradients (brute force), closed forms (homogeneous RVE, exact laminate), Hill-Mandel
(Eq. Hill-Mandel), dPbar/dFbar by finite differences, quadratic Newton convergence, Voigt/Reuss
bounds, objectivity, the paper's literal B^T CC B + G_hat tangent and its T-matrix stiffness
transfer (Eq. k-mac-element-6)."""
import numpy as np
import pytest

import synth
from oracle import material as mat
from oracle.rve import PeriodicRVE


def circle_rve(n, ratio=10.0, r=0.25, center=(0.5, 0.5)):
    return PeriodicRVE(n, 2, synth.phase_from_inclusions(n, 2, [center], [r]), [1.0, ratio], [0.3, 0.3])


def sphere_rve(n, ratio=10.0, phi=0.2):
    return PeriodicRVE(n, 3, synth.sphere_rve(n, 1, phi, [[0.45, 0.5, 0.55]]), [1.0, ratio], [0.3, 0.3])


def total_energy(rve, w, Fbar):
    F = rve.F_at_qps(w, Fbar)
    return rve.wdet * mat.psi(F, rve.lam_e[:, None], rve.mu_e[:, None]).sum()


@pytest.mark.parametrize("d,n", [(2, 3), (3, 2)])
def test_residual_is_energy_gradient_bruteforce(d, n):
    ph = (synth.uniform(5, np.arange(n ** d), 1)[:, 0] > 0.5).astype(np.uint8)
    rve = PeriodicRVE(n, d, ph, [1.0, 5.0], [0.3, 0.25])
    Fbar = synth.random_F(21, 1, d, 0.1)[0]
    w = synth.random_field(22, 1, rve.n_dof, 0.02)[0]
    R, _ = rve.residual(w, Fbar)
    h = 1e-6
    fd = np.zeros(rve.n_dof)
    for k in range(rve.n_dof):
        e = np.zeros(rve.n_dof)
        e[k] = h
        fd[k] = (total_energy(rve, w + e, Fbar) - total_energy(rve, w - e, Fbar)) / (2 * h)
    np.testing.assert_allclose(R, fd, atol=1e-9)
    K = rve.tangent(w, Fbar).toarray()
    Kfd = np.zeros_like(K)
    for k in range(rve.n_dof):
        e = np.zeros(rve.n_dof)
        e[k] = h
        Kfd[:, k] = (rve.residual(w + e, Fbar)[0] - rve.residual(w - e, Fbar)[0]) / (2 * h)
    np.testing.assert_allclose(K, Kfd, atol=1e-7 * np.abs(K).max())


@pytest.mark.parametrize("d", [2, 3])
def test_tangent_equals_paper_literal_form(d):
    rve = circle_rve(4) if d == 2 else sphere_rve(3)
    Fbar = synth.random_F(23, 1, d, 0.1)[0]
    w = synth.random_field(24, 1, rve.n_dof, 0.01)[0]
    K1 = rve.tangent(w, Fbar)
    K2 = rve.tangent_literal(w, Fbar)
    assert abs(K1 - K2).max() < 1e-12 * abs(K1).max()


@pytest.mark.parametrize("d", [2, 3])
def test_homogeneous_rve_is_closed_form(d):
    n = 4 if d == 2 else 3
    rve = PeriodicRVE(n, d, np.zeros(n ** d, np.uint8), [3.0, 3.0], [0.3, 0.3])
    Fbar = synth.random_F(25, 1, d, 0.15)[0]
    out = rve.solve(Fbar, synth.random_field(26, 1, rve.n_dof, 0.01)[0], rtol=1e-14)
    lam, mu = mat.lame(3.0, 0.3)
    np.testing.assert_allclose(out["w"], 0, atol=1e-12)
    np.testing.assert_allclose(out["P"], mat.P_of_F(Fbar, lam, mu), atol=1e-13)
    np.testing.assert_allclose(out["A"], mat.A_of_F(Fbar, lam, mu), atol=1e-12)
    np.testing.assert_allclose(out["W"], mat.psi(Fbar, lam, mu), atol=1e-14)


def test_uniaxial_closed_form_on_homogeneous_rve():
    lam, mu = mat.lame(1.0, 0.3)
    s = 1.1
    t = np.sqrt((lam / 2 + mu) / (lam * s * s / 2 + mu))
    rve = PeriodicRVE(8, 2, np.zeros(64, np.uint8), [1.0, 1.0], [0.3, 0.3])
    out = rve.solve(np.diag([s, t]))
    assert abs(out["P"][1, 1]) < 1e-14
    assert abs(out["P"][0, 0] - s * (lam / 2 * (s * s * t * t - 1) / (s * s) + mu * (1 - 1 / (s * s)))) < 1e-14


def laminate_exact(Fbar, phis, lams, mus, N):
    """Rank-one laminate: F_i = Fbar + a_i (x) N, sum phi_i a_i = 0, P(F_0) N = P(F_1) N, solved by
    Newton with finite-difference Jacobian (independent of the FE code)."""
    d = Fbar.shape[0]
    a = np.zeros(d)

    def g(a):
        a1 = -phis[0] / phis[1] * a
        F0 = Fbar + np.outer(a, N)
        F1 = Fbar + np.outer(a1, N)
        return mat.P_of_F(F0, lams[0], mus[0]) @ N - mat.P_of_F(F1, lams[1], mus[1]) @ N

    for _ in range(50):
        r = g(a)
        if np.linalg.norm(r) < 1e-15:
            break
        Jm = np.zeros((d, d))
        for k in range(d):
            e = np.zeros(d)
            e[k] = 1e-7
            Jm[:, k] = (g(a + e) - g(a - e)) / 2e-7
        a = a - np.linalg.solve(Jm, r)
    a1 = -phis[0] / phis[1] * a
    F0, F1 = Fbar + np.outer(a, N), Fbar + np.outer(a1, N)
    return phis[0] * mat.P_of_F(F0, lams[0], mus[0]) + phis[1] * mat.P_of_F(F1, lams[1], mus[1])


@pytest.mark.parametrize("d", [2, 3])
def test_laminate_exact_solution(d):
    n = 8 if d == 2 else 4
    layer = np.arange(n) < (3 if d == 2 else 1)  # rows j (2D) / planes k (3D) of phase 1
    idx = np.arange(n ** d)
    last = idx // n ** (d - 1)
    ph = layer[last].astype(np.uint8)
    E, nu = [1.0, 7.0], [0.3, 0.2]
    rve = PeriodicRVE(n, d, ph, E, nu)
    lam, mu = mat.lame(np.array(E), np.array(nu))
    phis = [1 - ph.mean(), ph.mean()]
    N = np.zeros(d)
    N[-1] = 1.0
    Fbar = synth.random_F(27, 1, d, 0.15)[0]
    out = rve.solve(Fbar, rtol=1e-14)
    P_ex = laminate_exact(Fbar, phis, lam, mu, N)
    np.testing.assert_allclose(out["P"], P_ex, atol=5e-13)
    h = 1e-5
    for k in range(d):
        for l in range(d):
            E_ = np.zeros((d, d))
            E_[k, l] = h
            fd = (laminate_exact(Fbar + E_, phis, lam, mu, N) - laminate_exact(Fbar - E_, phis, lam, mu, N)) / (2 * h)
            np.testing.assert_allclose(out["A"][:, :, k, l], fd, atol=2e-8)


def bad_start(n, d, amp=0.8):
    """A fluctuation that folds the elements next to node 1 (dw_x/dX_1 about -amp*n near it)."""
    w = np.zeros(d * n ** d)
    w[d * 1 + 0] = amp
    return w


@pytest.mark.parametrize("d", [2, 3])
def test_load_continuation_reaches_the_laminate_closed_form(d):
    """Continuation from w = 0 in equal increments of Fbar - I lands on the exact laminate
    solution, from a start state the plain Newton iteration rejects (J <= 0)."""
    from oracle.rve import STATUS_J_NONPOS
    n = 4
    ph = (np.arange(n ** d) // n ** (d - 1) < 1).astype(np.uint8)
    E, nu = [1.0, 7.0], [0.3, 0.2]
    rve = PeriodicRVE(n, d, ph, E, nu)
    lam, mu = mat.lame(np.array(E), np.array(nu))
    Fbar = synth.random_F(29, 1, d, 0.2)[0]
    w_bad = bad_start(n, d)
    assert rve.newton(Fbar, w_bad)[1] == STATUS_J_NONPOS
    out = rve.solve(Fbar, w_bad, rtol=1e-14, stages=4)
    assert out["status"] == 0
    N = np.zeros(d)
    N[-1] = 1.0
    np.testing.assert_allclose(out["P"], laminate_exact(Fbar, [1 - ph.mean(), ph.mean()], lam, mu, N), atol=5e-13)
    direct = rve.solve(Fbar, rtol=1e-14)
    np.testing.assert_allclose(out["A"], direct["A"], atol=1e-11)


@pytest.fixture(scope="module")
def solved2d():
    rve = circle_rve(8, ratio=10.0, r=0.3, center=(0.4, 0.55))
    Fbar = np.array([[1.12, 0.07], [-0.03, 0.93]])
    return rve, Fbar, rve.solve(Fbar, rtol=1e-14)


def test_quadratic_newton_convergence(solved2d):
    _, _, out = solved2d
    h = out["history"]
    assert out["status"] == 0 and out["newton_iters"] <= 6
    # last steps before the round-off floor: r_{k+1} <= C r_k^2
    pairs = [(a, b) for a, b in zip(h[:-1], h[1:]) if a > 1e-8 and a < 1e-2]
    assert pairs, h
    for a, b in pairs:
        assert b <= 50.0 * a * a, h


def test_hill_mandel_and_mean_F(solved2d):
    rve, Fbar, out = solved2d
    np.testing.assert_allclose(out["F_mean"], Fbar, atol=1e-14)
    F = rve.F_at_qps(out["w"], Fbar)
    P = mat.P_of_F(F, rve.lam_e[:, None], rve.mu_e[:, None])
    PF = rve.wdet * np.einsum("eqiJ,eqiJ->", P, F)
    assert abs(PF - np.sum(out["P"] * Fbar)) < 1e-12
    dw = synth.random_field(31, 1, rve.n_dof, 1.0)[0]
    dF = rve.F_at_qps(dw, np.zeros((2, 2)))
    assert abs(rve.wdet * np.einsum("eqiJ,eqiJ->", P, dF)) < 1e-12


def test_P_is_derivative_of_W_and_A_of_P(solved2d):
    rve, Fbar, out = solved2d
    h = 1e-5
    for k in range(2):
        for l in range(2):
            E = np.zeros((2, 2))
            E[k, l] = h
            p = rve.solve(Fbar + E, out["w"], rtol=1e-14)
            m = rve.solve(Fbar - E, out["w"], rtol=1e-14)
            assert abs((p["W"] - m["W"]) / (2 * h) - out["P"][k, l]) < 1e-9
            np.testing.assert_allclose((p["P"] - m["P"]) / (2 * h), out["A"][:, :, k, l], atol=1e-8)


def test_objectivity_of_homogenised_response(solved2d):
    rve, Fbar, out = solved2d
    c, s = np.cos(0.4), np.sin(0.4)
    Q = np.array([[c, -s], [s, c]])
    rot = rve.solve(Q @ Fbar, out["w"] @ np.kron(np.eye(rve.n_nodes), Q.T), rtol=1e-14)
    np.testing.assert_allclose(rot["W"], out["W"], rtol=1e-12)
    np.testing.assert_allclose(rot["P"], Q @ out["P"], atol=1e-12)


def mandel(C4):
    d = C4.shape[0]
    pairs = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    wgt = [1.0 if i == j else np.sqrt(2.0) for i, j in pairs]
    return np.array([[C4[i, j, k, l] * wgt[p] * wgt[q] for q, (k, l) in enumerate(pairs)]
                     for p, (i, j) in enumerate(pairs)])


@pytest.mark.parametrize("d", [2, 3])
def test_small_strain_between_voigt_and_reuss(d):
    rve = circle_rve(8, 20.0) if d == 2 else sphere_rve(4, 20.0, 0.25)
    out = rve.solve(np.eye(d))
    Ceff = mandel(out["A"])
    lam, mu = mat.lame(np.array([1.0, 20.0]), np.array([0.3, 0.3]))
    phi1 = rve.phase.mean()
    C0, C1 = mandel(mat.hooke(lam[0], mu[0], d)), mandel(mat.hooke(lam[1], mu[1], d))
    CV = (1 - phi1) * C0 + phi1 * C1
    CR = np.linalg.inv((1 - phi1) * np.linalg.inv(C0) + phi1 * np.linalg.inv(C1))
    eps = synth.random_field(41, 20, CV.shape[0], 1.0)
    for e in eps:
        eff = e @ Ceff @ e
        assert e @ CR @ e <= eff * (1 + 1e-12)
        assert eff <= e @ CV @ e * (1 + 1e-12)
    # the upper bound is strict for a heterogeneous cell
    assert np.trace(Ceff) < np.trace(CV)


@pytest.mark.parametrize("d", [2, 3])
def test_condensation_equals_paper_T_matrix_transfer(d):
    rve = circle_rve(6) if d == 2 else sphere_rve(3)
    Fbar = synth.random_F(51, 1, d, 0.1)[0]
    out = rve.solve(Fbar, rtol=1e-14)
    nen = 2 ** d
    from oracle.rve import corner_offsets
    s = 2.0 * corner_offsets(d) - 1.0
    xi = np.full(d, 0.2)
    Nval = np.prod((1 + s * xi) / 2, axis=1)
    gradN = np.stack([s[:, m] / 2 * np.prod(np.delete((1 + s * xi) / 2, m, axis=1), axis=1) for m in range(d)], 1)
    k_T = rve.stiffness_transfer_T(out["w"], Fbar, gradN, Nval, omega=0.7)
    k_A = 0.7 * np.einsum("IL,iLjN,JN->IiJj", gradN, out["A"], gradN).reshape(nen * d, nen * d)
    np.testing.assert_allclose(k_T, k_A, atol=1e-12 * np.abs(k_A).max())
