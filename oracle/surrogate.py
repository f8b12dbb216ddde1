"""FP64 reference of the surrogate constitutive map (oracle; test infrastructure only).

W(F) = W_base(C) + sg * y(x), C = F^T F, x = Mandel(E)/sx, E = (C - I)/2, with W_base the
compressible neo-Hookean law of oracle.material at (lam0, mu0) and y the MLP of oracle.mlp.
P = dW/dF and A = dP/dF follow by the chain rule:
  S = S_base + (sg/sx) sum_p g_p dx_p/dE (Mandel weights), CC = CC_base + (sg/sx^2) (Mandel H),
  P = F S, A_iJkL = delta_ik S_JL + F_iI F_kK CC_IJKL.
The correction may carry a polynomial part y_poly(x) = sum_a c_a x^n(a) over the monomials of
degree 3 to 6 (each degree's nondecreasing index tuples in lexicographic order), evaluated here
from exponent vectors n by the power rule.
Pinned by central finite differences of W(F) and P(F) in tests/test_oracle_mlp.py.
Trust measure: |U - I|_F with U = C^(1/2) from numpy's symmetric eigen-decomposition.
"""
from __future__ import annotations

import itertools

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


def poly_exponents():
    """Exponent vectors (896, 6) of the monomials of degree 3, 4, 5, 6 in 6 variables, in the order
    of the coefficients: per degree, the nondecreasing index tuples in lexicographic order."""
    rows = []
    for d in (3, 4, 5, 6):
        for tup in itertools.combinations_with_replacement(range(6), d):
            rows.append(np.bincount(np.array(tup), minlength=6))
    return np.array(rows)


def _pow(x, n):
    """x^n elementwise with 0^0 = 1 and x^(negative) = 0 (the derivative of a missing factor)."""
    out = np.where(n >= 0, np.abs(x) ** np.maximum(n, 0) * np.sign(x) ** np.maximum(n, 0), 0.0)
    return np.where(n == 0, 1.0, out)


def poly_value_grad_hess(coef, x):
    """y_poly, its gradient and Hessian at features x (m, 6) by the power rule on exponent
    vectors: d x^n / dx_k = n_k x^(n - e_k), d2 x^n / dx_k dx_l = n_k (n_l - delta_kl) x^(n - e_k - e_l)."""
    coef = np.asarray(coef, dtype=np.float64)
    N = poly_exponents()
    x = np.asarray(x, dtype=np.float64)
    m = x.shape[0]
    E6 = np.eye(6, dtype=int)

    def mono(n):  # (m, terms) values of x^n for exponent rows n (terms, 6)
        return np.prod(_pow(x[:, None, :], n[None, :, :]), axis=-1)

    y = mono(N) @ coef
    g = np.zeros((m, 6))
    H = np.zeros((m, 6, 6))
    for k in range(6):
        nk = N[:, k].astype(np.float64)
        g[:, k] = mono(N - E6[k]) @ (coef * nk)
        for l in range(6):
            fac = nk * (N[:, l] - (1 if k == l else 0))
            H[:, k, l] = mono(N - E6[k] - E6[l]) @ (coef * fac)
    return y, g, H


def evaluate(params, F, lam0, mu0, sx, sg, bf16=False, Ca=None, origin=None, poly=None):
    """W, P, A at deformation gradients F (..., 3, 3).  Ca (6x6 Mandel, optional): anisotropic
    quadratic base term 1/2 m(E).Ca.m(E), m(E) the Mandel vector of E.  origin = (y0, g0, H0)
    (optional): the network's Taylor terms at x = 0, subtracted from the correction.  poly
    (896 coefficients, optional): the polynomial part of the correction (see poly_exponents)."""
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
    if poly is not None:
        yp, gp, Hp = poly_value_grad_hess(poly, x)
        y = y + yp.reshape(shp)
        g = g + gp.reshape(shp + (6,))
        H = H + Hp.reshape(shp + (6, 6))
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
