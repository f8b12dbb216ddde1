"""RVE with kinematic uniform boundary conditions (KUBC), FP64 (oracle; test infrastructure only).

The paper's RVE coupling is periodic; Sec. 3.2 lists kinematically uniform (Dirichlet) boundary
conditions among the energetically consistent choices, and Sec. 4 (Eq. ModelingError) gives
their modelling error, of order epsilon/delta from boundary layers, where periodic coupling has
none.  With KUBC the boundary of the sampling domain follows the linearised macro field exactly:
u = (Fbar - I) X on the boundary, so the fluctuation w vanishes there and only interior nodes
are free.  Everything else is as in
`rve.PeriodicRVE`: Q1/Hex8 elements with full Gauss integration on the unit cell, F = Fbar +
Grad w, the residual R_a = sum wt detJ P Grad N_a on the interior nodes, Newton with sparse LU,
Pbar = <P>, Wbar = <psi>, and the tangent transfer by static condensation Abar = <A> -
L^T K^-1 L over the interior dofs.

Pins (tests/test_oracle_kubc.py): homogeneous RVE = pointwise law; Pbar = dWbar/dFbar and
Abar = dPbar/dFbar by finite differences; Hill-Mandel; Hill's ordering of the small-strain
tangents Voigt >= KUBC >= periodic >= Reuss; KUBC on k x k tilings of one cell decreasing
towards the periodic value.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import material as mat
from .rve import STATUS_J_NONPOS, STATUS_NEWTON_CAP, STATUS_NONFINITE, STATUS_OK, corner_offsets, gauss_points, \
    shape_and_grad


class DirichletRVE:
    """One microstructure on an n^d element grid of the unit cell, (n+1)^d nodes, w = 0 on the
    boundary nodes."""

    def __init__(self, n, dim, phase, E, nu):
        self.n, self.d = int(n), int(dim)
        d, n = self.d, self.n
        self.phase = np.asarray(phase, dtype=np.int64).reshape(-1)
        assert self.phase.size == n ** d
        lam, mu = mat.lame(np.asarray(E, dtype=np.float64), np.asarray(nu, dtype=np.float64))
        self.lam_e, self.mu_e = lam[self.phase], mu[self.phase]
        m = n + 1
        self.n_nodes = m ** d
        self.n_dof = self.n_nodes * d
        self.h = 1.0 / n
        idx = np.array(list(itertools.product(range(n), repeat=d)))[:, ::-1]  # element (i, j[, k])
        off = corner_offsets(d)
        self.conn = ((idx[:, None, :] + off[None, :, :]) * m ** np.arange(d)).sum(-1)  # (n_el, nen)
        nodes = np.array(list(itertools.product(range(m), repeat=d)))[:, ::-1]  # node (i, j[, k])
        boundary = ((nodes == 0) | (nodes == n)).any(axis=1)
        self.free = np.nonzero(np.repeat(~boundary, d))[0]
        self.X = nodes * self.h
        xi = gauss_points(d)
        self.N, self.G = shape_and_grad(d, xi, np.full(d, self.h))
        self.wdet = (self.h / 2.0) ** d

    def F_at_qps(self, w, Fbar):
        we = w.reshape(self.n_nodes, self.d)[self.conn]
        return Fbar[None, None] + np.einsum("eai,qaJ->eqiJ", we, self.G)

    def residual(self, w, Fbar):
        F = self.F_at_qps(w, Fbar)
        P = mat.P_of_F(F, self.lam_e[:, None], self.mu_e[:, None])
        Re = self.wdet * np.einsum("eqiJ,qaJ->eai", P, self.G)
        R = np.zeros((self.n_nodes, self.d))
        np.add.at(R, self.conn, Re)
        return R.reshape(-1), F

    def tangent(self, w, Fbar):
        F = self.F_at_qps(w, Fbar)
        A = mat.A_of_F(F, self.lam_e[:, None], self.mu_e[:, None])
        ke = self.wdet * np.einsum("qaJ,eqiJkL,qbL->eaibk", self.G, A, self.G)
        nen, d = self.G.shape[1], self.d
        dofs = (self.conn[:, :, None] * d + np.arange(d)[None, None, :]).reshape(self.conn.shape[0], -1)
        rows = np.repeat(dofs, nen * d, axis=1).reshape(-1)
        cols = np.tile(dofs, (1, nen * d)).reshape(-1)
        return sp.csr_matrix((ke.reshape(-1), (rows, cols)), shape=(self.n_dof, self.n_dof))

    def newton(self, Fbar, rtol=1e-12, atol=1e-14, max_iter=30):
        Fbar = np.asarray(Fbar, dtype=np.float64)
        w = np.zeros(self.n_dof)
        R, F = self.residual(w, Fbar)
        if np.any(np.linalg.det(F) <= 0):
            return w, STATUS_J_NONPOS, 0
        r0 = float(np.linalg.norm(R[self.free]))
        rn, it = r0, 0
        while True:
            if not np.isfinite(rn):
                return w, STATUS_NONFINITE, it
            if rn <= max(rtol * r0, atol):
                return w, STATUS_OK, it
            if it >= max_iter:
                return w, STATUS_NEWTON_CAP, it
            K = self.tangent(w, Fbar)
            w[self.free] += spla.spsolve(K[self.free][:, self.free].tocsc(), -R[self.free])
            it += 1
            R, F = self.residual(w, Fbar)
            if np.any(np.linalg.det(F) <= 0):
                return w, STATUS_J_NONPOS, it
            rn = float(np.linalg.norm(R[self.free]))

    def averages(self, w, Fbar):
        """<P>, <F>, <psi>, <A> over the cell (|Omega| = 1)."""
        F = self.F_at_qps(w, Fbar)
        lam, mu = self.lam_e[:, None], self.mu_e[:, None]
        s = self.wdet
        return (s * mat.P_of_F(F, lam, mu).sum(axis=(0, 1)), s * F.sum(axis=(0, 1)),
                s * mat.psi(F, lam, mu).sum(), s * mat.A_of_F(F, lam, mu).sum(axis=(0, 1)))

    def condensed_tangent(self, w, Fbar):
        """Abar = <A> - L_f^T K_ff^-1 L_f over the interior dofs, L = dR/dFbar."""
        d = self.d
        _, _, _, Am = self.averages(w, Fbar)
        F = self.F_at_qps(w, Fbar)
        A = mat.A_of_F(F, self.lam_e[:, None], self.mu_e[:, None])
        Le = self.wdet * np.einsum("qaJ,eqiJkL->eaikL", self.G, A)
        L = np.zeros((self.n_nodes, d, d, d))
        np.add.at(L, self.conn, Le)
        L = L.reshape(self.n_dof, d * d)[self.free]
        K = self.tangent(w, Fbar)[self.free][:, self.free].tocsc()
        X = spla.spsolve(K, L)
        X = X.reshape(-1, d * d) if X.ndim == 1 else X
        return Am - (L.T @ X).reshape(d, d, d, d)

    def solve(self, Fbar, rtol=1e-12, atol=1e-14, max_iter=30, tangent=True):
        w, status, it = self.newton(Fbar, rtol, atol, max_iter)
        out = {"w": w, "status": status, "newton_iters": it}
        if status in (STATUS_OK, STATUS_NEWTON_CAP):
            P, Fm, W, _ = self.averages(w, np.asarray(Fbar, dtype=np.float64))
            out.update(P=P, F_mean=Fm, W=W)
            if tangent:
                out["A"] = self.condensed_tangent(w, np.asarray(Fbar, dtype=np.float64))
        return out
