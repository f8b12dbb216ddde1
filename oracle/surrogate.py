"""FP64 reference of the surrogate constitutive map (oracle; test infrastructure only).

W(F) = W_base(C) + sg * y(x), C = F^T F, x = Mandel(E)/sx, E = (C - I)/2, with W_base the
compressible neo-Hookean law of oracle.material at (lam0, mu0) and y the MLP of oracle.mlp.
P = dW/dF and A = dP/dF follow by the chain rule:
  S = S_base + (sg/sx) sum_p g_p dx_p/dE (Mandel weights), CC = CC_base + (sg/sx^2) (Mandel H),
  P = F S, A_iJkL = delta_ik S_JL + F_iI F_kK CC_IJKL.
Pinned by central finite differences of W(F) and P(F) in tests/test_oracle_mlp.py.
Trust measure: |U - I|_F with U = C^(1/2) from numpy's symmetric eigen-decomposition.
"""
from __future__ import annotations

import numpy as np

from . import material as mat
from . import mlp

MANDEL = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
WMAN = np.array([1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)])


def features(F, sx):
    C = np.swapaxes(F, -1, -2) @ F
    E = 0.5 * (C - np.eye(3))
    return np.stack([E[..., i, j] for i, j in MANDEL], -1) * WMAN / sx


def stretch_distance(F):
    C = np.swapaxes(F, -1, -2) @ F
    lam = np.linalg.eigvalsh(C)
    return np.sqrt(((np.sqrt(lam) - 1.0) ** 2).sum(-1))


def _to_tensor2(v):
    """Symmetric tensors from Mandel-weighted vectors divided by w_p: T_IJ = v_p / w_p."""
    T = np.zeros(v.shape[:-1] + (3, 3))
    for p, (i, j) in enumerate(MANDEL):
        T[..., i, j] = T[..., j, i] = v[..., p] / WMAN[p]
    return T


def _to_tensor4(H):
    CC = np.zeros(H.shape[:-2] + (3, 3, 3, 3))
    for p, (i, j) in enumerate(MANDEL):
        for q, (k, l) in enumerate(MANDEL):
            v = H[..., p, q] / (WMAN[p] * WMAN[q])
            for a, b in {(i, j), (j, i)}:
                for c, d in {(k, l), (l, k)}:
                    CC[..., a, b, c, d] = v
    return CC


def evaluate(params, F, lam0, mu0, sx, sg, bf16=False, Ca=None, origin=None):
    """W, P, A at deformation gradients F (..., 3, 3).  Ca (6x6 Mandel, optional): anisotropic
    quadratic base term 1/2 m(E).Ca.m(E), m(E) the Mandel vector of E.  origin = (y0, g0, H0)
    (optional): the network's Taylor terms at x = 0, subtracted from the correction."""
    F = np.asarray(F, dtype=np.float64)
    x = features(F, sx).reshape(-1, 6)
    y, g, H = mlp.input_hessian(params, x, bf16)
    shp = F.shape[:-2]
    y, g, H = y.reshape(shp), g.reshape(shp + (6,)), H.reshape(shp + (6, 6))
    if origin is not None:
        y0, g0, H0 = (np.asarray(v, dtype=np.float64) for v in origin)
        xs = x.reshape(shp + (6,))
        hx = xs @ H0.T
        y = y - y0 - (xs * g0).sum(-1) - 0.5 * (xs * hx).sum(-1)
        g = g - g0 - hx
        H = H - H0
    C = np.swapaxes(F, -1, -2) @ F
    Wb = mat.psi(F, lam0, mu0)
    S = mat.S_of_C(C, lam0, mu0) + sg / sx * _to_tensor2(g)
    CC = mat.CC_of_C(C, lam0, mu0) + sg / sx ** 2 * _to_tensor4(H)
    if Ca is not None:
        m = features(F, 1.0)  # Mandel vector of E
        sm = m @ np.asarray(Ca).T
        Wb = Wb + 0.5 * (m * sm).sum(-1)
        S = S + _to_tensor2(sm)
        CC = CC + _to_tensor4(np.broadcast_to(np.asarray(Ca), sm.shape[:-1] + (6, 6)))
    P = F @ S
    A = np.einsum("ik,...JL->...iJkL", np.eye(3), S) + np.einsum("...iI,...kK,...IJKL->...iJkL", F, F, CC)
    return Wb + sg * y, P, A
