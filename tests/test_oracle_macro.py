"""Pins of the oracle's macro FE-HMM layer: energy consistency of the assembled residual and
tangent (finite differences), the S^H route of Eq. f_I^int / macro-mean-stress, the patch test on
the structured mesh, and an end-to-end nested load-step run on a homogeneous microstructure whose
macro solution has the uniaxial closed form."""
import numpy as np
import pytest

import synth
from oracle import driver
from oracle import material as mat
from oracle.macro import MacroMesh


@pytest.mark.parametrize("n", [(3, 2), (2, 2, 1)])
def test_assembly_is_energy_gradient(n):
    d = len(n)
    mesh = MacroMesh(n)
    lam, mu = mat.lame(2.0, 0.3)
    u = synth.random_field(61, 1, mesh.n_dof, 0.05)[0]

    def energy(u):
        return mesh.omega * mat.psi(mesh.qp_F(u), lam, mu).sum()

    F = mesh.qp_F(u)
    f, K = mesh.assemble(mat.P_of_F(F, lam, mu), mat.A_of_F(F, lam, mu))
    h = 1e-6
    for k in range(0, mesh.n_dof, 3):
        e = np.zeros(mesh.n_dof)
        e[k] = h
        assert abs((energy(u + e) - energy(u - e)) / (2 * h) - f[k]) < 1e-9
        Fp, Fm = mesh.qp_F(u + e), mesh.qp_F(u - e)
        fp, _ = mesh.assemble(mat.P_of_F(Fp, lam, mu), mat.A_of_F(Fp, lam, mu))
        fm, _ = mesh.assemble(mat.P_of_F(Fm, lam, mu), mat.A_of_F(Fm, lam, mu))
        np.testing.assert_allclose(K[:, k].toarray()[:, 0], (fp - fm) / (2 * h), atol=1e-8)
    np.testing.assert_allclose(mesh.assemble_f_via_S(mat.P_of_F(F, lam, mu), F), f, atol=1e-13)


@pytest.mark.parametrize("n", [(4, 3), (2, 3, 2)])
def test_patch_test_affine_field(n):
    d = len(n)
    mesh = MacroMesh(n)
    H = synth.random_F(62, 1, d, 0.1)[0] - np.eye(d)
    u = (mesh.X @ H.T).reshape(-1)
    F = mesh.qp_F(u)
    np.testing.assert_allclose(F, np.broadcast_to(np.eye(d) + H, F.shape), atol=1e-14)
    lam, mu = mat.lame(1.0, 0.3)
    f, _ = mesh.assemble(mat.P_of_F(F, lam, mu), mat.A_of_F(F, lam, mu))
    boundary = (np.isclose(mesh.X, 0) | np.isclose(mesh.X, 1)).any(1)
    interior = np.repeat(~boundary, d)
    np.testing.assert_allclose(f[interior], 0, atol=1e-14)


def test_nested_run_homogeneous_config1_closed_form():
    """The 4x4 Q1 uniaxial boundary conditions with a homogeneous microstructure: the macro solution is the
    uniaxial plane-strain state F = diag(s, t), t^2 = (lam/2 + mu)/(lam s^2/2 + mu)."""
    p = synth.uniaxial_2d_small()
    p.rve_E[:] = 1.0
    recs, mesh = driver.run(p, n_steps=10, steps_to_run=3)
    lam, mu = mat.lame(1.0, 0.3)
    for r in recs:
        s = 1.0 + 0.1 * r["step"] / 10
        t = np.sqrt((lam / 2 + mu) / (lam * s * s / 2 + mu))
        top = np.isclose(mesh.X[:, 1], 1.0)
        np.testing.assert_allclose(r["u"].reshape(-1, 2)[top, 1], t - 1.0, atol=1e-12)
        np.testing.assert_allclose(r["P"][:, 1, 1], 0, atol=1e-12)
        assert r["converged"]


def test_nested_and_alternating_reach_same_state():
    """Both schemes satisfy the same discrete equations at the end of a load step (Sec. 5)."""
    p = synth.uniaxial_2d_small()
    nested, _ = driver.run(p, scheme="nested", steps_to_run=2)
    alt, _ = driver.run(p, scheme="alternating", steps_to_run=2)
    for a, b in zip(nested, alt):
        np.testing.assert_allclose(a["u"], b["u"], atol=1e-9)
        np.testing.assert_allclose(a["P"], b["P"], atol=1e-9)
