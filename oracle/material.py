"""Compressible neo-Hookean hyperelasticity in FP64 (oracle; test infrastructure only).

Follows Sec. 6 of the paper: Eq. (NH-free-energy) for psi, the closed forms for
S = 2 dpsi/dC and CC = 4 d2psi/dCdC, and Eq. (Aijkl-NeoHook) for dC^-1/dC.  The
first Piola-Kirchhoff stress P = F S and its tangent dP/dF follow from the
hyperelastic relations of Eq. (hyperelasticity-PF).

2D is plane strain: F_33 = 1, so C is block diagonal with C_33 = 1,
tr C - 3 = C_11 + C_22 - 2 and J = det of the in-plane 2x2 block.  All
functions broadcast over leading axes; F has shape (..., d, d).
"""
from __future__ import annotations

import numpy as np


def lame(E, nu):
    """Lame constants from Young's modulus and Poisson ratio (the conversion behind the
    paper's Table of material parameters, Sec. 6)."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def _trC_minus_3(C):
    d = C.shape[-1]
    tr = np.trace(C, axis1=-2, axis2=-1)
    return tr - 3.0 if d == 3 else tr + 1.0 - 3.0  # plane strain adds C_33 = 1


def psi(F, lam, mu):
    """Free energy, Eq. (NH-free-energy): lam/4 (J^2-1) - (lam/2+mu) ln J + mu/2 (tr C - 3)."""
    F = np.asarray(F, dtype=np.float64)
    J = np.linalg.det(F)
    C = np.swapaxes(F, -1, -2) @ F
    return lam / 4.0 * (J * J - 1.0) - (lam / 2.0 + mu) * np.log(J) + mu / 2.0 * _trC_minus_3(C)


def S_of_C(C, lam, mu):
    """Second Piola-Kirchhoff stress: S = lam/2 (J^2-1) C^-1 + mu (I - C^-1), J^2 = det C."""
    C = np.asarray(C, dtype=np.float64)
    d = C.shape[-1]
    Ci = np.linalg.inv(C)
    J2 = np.linalg.det(C)
    lam = np.asarray(lam)[..., None, None]
    mu = np.asarray(mu)[..., None, None]
    return lam / 2.0 * (J2[..., None, None] - 1.0) * Ci + mu * (np.eye(d) - Ci)


def dCinv_dC(Ci):
    """The paper's fourth-order tensor A_ijkl = -1/2 (Ci_ik Ci_jl + Ci_jk Ci_il), Eq. (Aijkl-NeoHook)."""
    return -0.5 * (np.einsum("...ik,...jl->...ijkl", Ci, Ci) + np.einsum("...jk,...il->...ijkl", Ci, Ci))


def CC_of_C(C, lam, mu):
    """Material tangent CC_ijkl = [lam (J^2-1) - 2 mu] A_ijkl + lam J^2 Ci_ij Ci_kl."""
    C = np.asarray(C, dtype=np.float64)
    Ci = np.linalg.inv(C)
    J2 = np.linalg.det(C)
    lam = np.asarray(lam)[..., None, None, None, None]
    mu = np.asarray(mu)[..., None, None, None, None]
    J2b = J2[..., None, None, None, None]
    return (lam * (J2b - 1.0) - 2.0 * mu) * dCinv_dC(Ci) + lam * J2b * np.einsum("...ij,...kl->...ijkl", Ci, Ci)


def P_of_F(F, lam, mu):
    """First Piola-Kirchhoff stress P = F S (Eq. hyperelasticity-PF: S = F^-1 P)."""
    F = np.asarray(F, dtype=np.float64)
    C = np.swapaxes(F, -1, -2) @ F
    return F @ S_of_C(C, lam, mu)


def A_of_F(F, lam, mu):
    """Nominal tangent A_iJkL = dP_iJ/dF_kL = delta_ik S_JL + F_iI F_kK CC_IJKL
    (the second derivative d2psi/dFdF of Eq. hyperelasticity-PF)."""
    F = np.asarray(F, dtype=np.float64)
    d = F.shape[-1]
    C = np.swapaxes(F, -1, -2) @ F
    S = S_of_C(C, lam, mu)
    CC = CC_of_C(C, lam, mu)
    geo = np.einsum("ik,...JL->...iJkL", np.eye(d), S)
    mat = np.einsum("...iI,...kK,...IJKL->...iJkL", F, F, CC)
    return geo + mat


def hooke(lam, mu, d):
    """Isotropic linear elasticity tensor lam 1x1 + 2 mu I^sym (textbook small-strain law)."""
    I = np.eye(d)
    return lam * np.einsum("ij,kl->ijkl", I, I) + mu * (np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I))


# ------------------------------------------------------------------ St. Venant-Kirchhoff
# The paper's second material case (Sec. 6, Table of material parameters, "linear elasticity
# along with geometrical nonlinearity"): the linear elastic law written in the Green-Lagrange
# strain E = (C - I)/2 and the second Piola-Kirchhoff stress,
#   psi = lam/2 (tr E)^2 + mu E:E,  S = lam tr(E) I + 2 mu E,  CC = lam I x I + 2 mu I^sym.
# Plane strain in 2D: E_33 = 0 (F_33 = 1), so tr E = E_11 + E_22.

def green_lagrange(F):
    F = np.asarray(F, dtype=np.float64)
    d = F.shape[-1]
    return 0.5 * (np.swapaxes(F, -1, -2) @ F - np.eye(d))


def svk_psi(F, lam, mu):
    E = green_lagrange(F)
    trE = np.trace(E, axis1=-2, axis2=-1)
    return lam / 2.0 * trE ** 2 + mu * np.einsum("...ij,...ij->...", E, E)


def svk_S(F, lam, mu):
    E = green_lagrange(F)
    d = E.shape[-1]
    trE = np.trace(E, axis1=-2, axis2=-1)[..., None, None]
    lam = np.asarray(lam)[..., None, None]
    mu = np.asarray(mu)[..., None, None]
    return lam * trE * np.eye(d) + 2.0 * mu * E


def svk_P(F, lam, mu):
    return np.asarray(F, dtype=np.float64) @ svk_S(F, lam, mu)


def svk_A(F, lam, mu):
    """dP_iJ/dF_kL = delta_ik S_JL + F_iI F_kK CC_IJKL with the constant CC of the law."""
    F = np.asarray(F, dtype=np.float64)
    d = F.shape[-1]
    S = svk_S(F, lam, mu)
    lam_b = np.asarray(lam)[..., None, None, None, None]
    mu_b = np.asarray(mu)[..., None, None, None, None]
    I = np.eye(d)
    CC = lam_b * np.einsum("IJ,KL->IJKL", I, I) + mu_b * (np.einsum("IK,JL->IJKL", I, I) + np.einsum("IL,JK->IJKL", I, I))
    geo = np.einsum("ik,...JL->...iJkL", I, S)
    return geo + np.einsum("...iI,...kK,...IJKL->...iJkL", F, F, CC)


# Constitutive laws by name: (psi, P, A).  "nh" is the paper's neo-Hookean law (Eq.
# NH-free-energy), "svk" the St. Venant-Kirchhoff law above.
LAWS = {"nh": (psi, P_of_F, A_of_F), "svk": (svk_psi, svk_P, svk_A)}
