"""Periodic RVE (micro problem) in FP64 (oracle; test infrastructure only).

The RVE is the unit cell [0,1]^d split into n^d Q1 (2D, plane strain) or Hex8
(3D) elements with full 2^d Gauss integration.  Following Sec. 3.2-3.3 of the
paper:

* Kinematics (Eq. linearization-uH with Eq. ConstraintCondition-phi_h-phi_H):
  u(X) = (Fbar - I) X + w(X) with w periodic, so F = Fbar + Grad w.  The
  periodic constraint matrix G of Eq. (ConstraintCondition-GtimesAlphaMinusBeta)
  is applied by identifying node n with node 0 on every axis; the Lagrange
  multipliers then drop out (G^T Lambda = 0 for periodic fields, Sec. 3.3).
  w at node 0 is pinned to 0 to remove the rigid translation (the paper asks for
  non-redundant constraints without naming the node).
* Residual (Eq. f_I^int, micro): R_a = sum_e sum_qp wt detJ P(F) Grad N_a, which
  equals int B^T S because P : Grad dv = S : dE (Sec. 2).
* Tangent (Eq. DG^h with Eq. G_IK-InitStressMatr, S_IK): K_ab,ik = sum wt detJ
  N_a,J A_iJkL N_b,L, the same bilinear form as B^T CC B + G_hat (checked in the
  tests against a literal B^T CC B + S_IK assembly).
* Newton (Eq. Saddlepoint-problem-Set-of-eqs, ch_3_eq_19-1, ch_3_eq_22):
  K dw = -R on the free dofs; w <- w + dw; stop on the 2-norm of R relative to
  the first residual of the solve, with an absolute floor.
* Averages (Eq. Average-of-P-and-F): Pbar = <P>, <F>, Wbar = <psi>.
* Tangent transfer: static condensation Abar = <A> - L^T K^-1 L with
  L = dR/dFbar, and, for cross-checking, the paper's literal transformation
  matrix form k^H = omega/|K_delta| T^T K T (Eq. k-mac-element-6/7) with T built
  from the saddle-point system ch_3_eq_30 on the non-periodic node grid.
The linear solves use scipy's sparse LU (a library primitive).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import material as mat

STATUS_OK, STATUS_NEWTON_CAP, STATUS_J_NONPOS, STATUS_NONFINITE = 0, 1, 2, 4


def corner_offsets(d):
    """Local node order: 2D (0,0),(1,0),(1,1),(0,1); 3D the same square at z=0 then z=1."""
    sq = [(0, 0), (1, 0), (1, 1), (0, 1)]
    if d == 2:
        return np.array(sq)
    return np.array([(a, b, c) for c in (0, 1) for (a, b) in sq])


def gauss_points(d):
    """2^d Gauss points in [-1,1]^d, lexicographic with xi_1 fastest; all weights 1."""
    g = 1.0 / math.sqrt(3.0)
    pts = [p[::-1] for p in itertools.product((-g, g), repeat=d)]
    return np.array(pts)


def shape_and_grad(d, xi, h):
    """Q1/Hex8 shape values N (nq, nen) and physical gradients G (nq, nen, d) on a cube of
    edge lengths h (array of d)."""
    off = corner_offsets(d)
    s = 2.0 * off - 1.0  # (nen, d) corner signs
    nq, nen = xi.shape[0], off.shape[0]
    N = np.ones((nq, nen))
    G = np.ones((nq, nen, d))
    for m in range(d):
        f = (1.0 + s[None, :, m] * xi[:, None, m]) / 2.0  # (nq, nen)
        N *= f
        for k in range(d):
            if k == m:
                G[:, :, k] *= s[None, :, m] / 2.0 * (2.0 / h[m])
            else:
                G[:, :, k] *= f
    return N, G


class PeriodicRVE:
    """One microstructure on a periodic n^d grid with per-element phases."""

    def __init__(self, n, dim, phase, E, nu, law="nh"):
        self.n, self.d = int(n), int(dim)
        self.law = law
        self._psi, self._P, self._A = mat.LAWS[law]
        d, n = self.d, self.n
        self.phase = np.asarray(phase, dtype=np.int64).reshape(-1)
        assert self.phase.size == n ** d
        lam, mu = mat.lame(np.asarray(E, dtype=np.float64), np.asarray(nu, dtype=np.float64))
        self.lam_e = lam[self.phase]
        self.mu_e = mu[self.phase]
        self.n_nodes = n ** d
        self.n_dof = self.n_nodes * d
        self.h = 1.0 / n
        # element connectivity (lexicographic element index, x fastest)
        idx = np.array(list(itertools.product(range(n), repeat=d)))[:, ::-1]  # (n_el, d): (i, j[, k])
        off = corner_offsets(d)
        self.elem_ijk = idx
        strides = n ** np.arange(d)
        self.conn = (((idx[:, None, :] + off[None, :, :]) % n) * strides).sum(-1)  # (n_el, nen)
        self.conn_np = ((idx[:, None, :] + off[None, :, :]) * (n + 1) ** np.arange(d)).sum(-1)
        xi = gauss_points(d)
        self.N, self.G = shape_and_grad(d, xi, np.full(d, self.h))
        self.wdet = (self.h / 2.0) ** d  # Gauss weight 1 times det J
        self.volume = 1.0
        self.free = np.arange(d, self.n_dof)  # node 0 pinned

    # ---------------------------------------------------------------- kinematics
    def F_at_qps(self, w, Fbar):
        """F = Fbar + Grad w at every Gauss point: shape (n_el, nq, d, d)."""
        we = w.reshape(self.n_nodes, self.d)[self.conn]  # (n_el, nen, d)
        return Fbar[None, None] + np.einsum("eai,qaJ->eqiJ", we, self.G)

    def _lam_mu(self):
        return self.lam_e[:, None], self.mu_e[:, None]

    # ------------------------------------------------------------------ residual
    def residual(self, w, Fbar):
        """R_a = sum_e sum_qp wt detJ P N_a,J  (flattened, n_dof)."""
        F = self.F_at_qps(w, Fbar)
        lam, mu = self._lam_mu()
        P = self._P(F, lam, mu)
        Re = self.wdet * np.einsum("eqiJ,qaJ->eai", P, self.G)
        R = np.zeros((self.n_nodes, self.d))
        np.add.at(R, self.conn, Re)
        return R.reshape(-1), F

    def element_tangents(self, w, Fbar):
        """Element matrices k_e[(a,i),(b,k)] = sum_qp wt detJ N_a,J A_iJkL N_b,L."""
        F = self.F_at_qps(w, Fbar)
        lam, mu = self._lam_mu()
        A = self._A(F, lam, mu)
        ke = self.wdet * np.einsum("qaJ,eqiJkL,qbL->eaibk", self.G, A, self.G)
        nen = self.G.shape[1]
        return ke.reshape(-1, nen * self.d, nen * self.d), A

    def _assemble(self, ke, conn, n_nodes):
        d = self.d
        dofs = (conn[:, :, None] * d + np.arange(d)[None, None, :]).reshape(conn.shape[0], -1)
        rows = np.repeat(dofs, dofs.shape[1], axis=1).reshape(-1)
        cols = np.tile(dofs, (1, dofs.shape[1])).reshape(-1)
        return sp.csr_matrix((ke.reshape(-1), (rows, cols)), shape=(n_nodes * d, n_nodes * d))

    def tangent(self, w, Fbar):
        ke, _ = self.element_tangents(w, Fbar)
        return self._assemble(ke, self.conn, self.n_nodes)

    def tangent_literal(self, w, Fbar):
        """The paper's form: k_T,IK = int (B_I^T CC B_K + G_hat_IK) with the Voigt B matrix of the
        Green-Lagrange strain and the initial-stress matrix G_hat_IK = S_IK 1 (Eq. DG^h, G_IK, S_IK).
        Used only to cross-check `tangent`."""
        d = self.d
        F = self.F_at_qps(w, Fbar)
        C = np.swapaxes(F, -1, -2) @ F
        lam, mu = self._lam_mu()
        if self.law == "svk":
            S = mat.svk_S(F, lam, mu)
            I = np.eye(d)
            lb, mb = lam[..., None, None, None, None], mu[..., None, None, None, None]
            CC = np.broadcast_to(lb * np.einsum("IJ,KL->IJKL", I, I)
                                 + mb * (np.einsum("IK,JL->IJKL", I, I) + np.einsum("IL,JK->IJKL", I, I)),
                                 F.shape[:2] + (d, d, d, d))
        else:
            S = mat.S_of_C(C, lam, mu)
            CC = mat.CC_of_C(C, lam, mu)
        pairs = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]
        nv = len(pairs)
        Cv = np.zeros(CC.shape[:2] + (nv, nv))
        for p, (I, J) in enumerate(pairs):
            for q, (K, L) in enumerate(pairs):
                Cv[..., p, q] = CC[..., I, J, K, L]
        nen = self.G.shape[1]
        B = np.zeros(F.shape[:2] + (nv, nen, d))  # dE_voigt / d(u_a,i)
        for p, (I, J) in enumerate(pairs):
            for a in range(nen):
                for i in range(d):
                    gI = self.G[None, :, a, I]
                    gJ = self.G[None, :, a, J]
                    if I == J:
                        B[..., p, a, i] = F[..., i, I] * gI
                    else:
                        B[..., p, a, i] = F[..., i, I] * gJ + F[..., i, J] * gI
        mat_part = np.einsum("eqpai,eqpr,eqrbk->eaibk", B, Cv, B)
        S_hat = np.einsum("qaI,eqIJ,qbJ->eab", self.G, S, self.G)  # S_IK of Eq. (S_IK)
        geo = S_hat[:, :, None, :, None] * np.eye(d)[None, None, :, None, :]
        ke = self.wdet * (mat_part + geo)
        return self._assemble(ke.reshape(-1, nen * d, nen * d), self.conn, self.n_nodes)

    # -------------------------------------------------------------------- Newton
    def newton(self, Fbar, w0=None, rtol=1e-10, atol=1e-14, max_iter=30, max_steps=None):
        """Newton iteration on the pinned periodic system.  `max_steps` caps the number of
        linear solves (1 gives the single micro iteration of Algorithm 2)."""
        Fbar = np.asarray(Fbar, dtype=np.float64)
        w = np.zeros(self.n_dof) if w0 is None else np.array(w0, dtype=np.float64)
        w[: self.d] = 0.0
        cap = max_iter if max_steps is None else max_steps
        R, F = self.residual(w, Fbar)
        if np.any(np.linalg.det(F) <= 0):
            return w, STATUS_J_NONPOS, 0, []
        r0 = float(np.linalg.norm(R[self.free]))
        hist = [r0]
        status, it = STATUS_NEWTON_CAP, 0
        while True:
            rn = hist[-1]
            if not np.isfinite(rn):
                status = STATUS_NONFINITE
                break
            if rn <= max(rtol * r0, atol):
                status = STATUS_OK
                break
            if it >= cap:
                status = STATUS_NEWTON_CAP if max_steps is None else STATUS_OK
                break
            K = self.tangent(w, Fbar)
            Kff = K[self.free][:, self.free].tocsc()
            dw = spla.spsolve(Kff, -R[self.free])
            w[self.free] += dw
            it += 1
            R, F = self.residual(w, Fbar)
            if np.any(np.linalg.det(F) <= 0):
                return w, STATUS_J_NONPOS, it, hist
            hist.append(float(np.linalg.norm(R[self.free])))
        return w, status, it, hist

    # ------------------------------------------------------------------ averages
    def averages(self, w, Fbar):
        """<P>, <F>, <psi> and <A> over the cell (Eq. Average-of-P-and-F); |Omega| = 1."""
        F = self.F_at_qps(w, Fbar)
        lam, mu = self._lam_mu()
        P = self._P(F, lam, mu)
        A = self._A(F, lam, mu)
        W = self._psi(F, lam, mu)
        s = self.wdet / self.volume
        return (s * P.sum(axis=(0, 1)), s * F.sum(axis=(0, 1)), s * W.sum(), s * A.sum(axis=(0, 1)))

    def dR_dFbar(self, w, Fbar):
        """L[(a,i),(k,L)] = sum wt detJ N_a,J A_iJkL: derivative of R with respect to Fbar."""
        F = self.F_at_qps(w, Fbar)
        lam, mu = self._lam_mu()
        A = self._A(F, lam, mu)
        Le = self.wdet * np.einsum("qaJ,eqiJkL->eaikL", self.G, A)
        L = np.zeros((self.n_nodes, self.d, self.d, self.d))
        np.add.at(L, self.conn, Le)
        return L.reshape(self.n_dof, self.d * self.d)

    def condensed_tangent(self, w, Fbar):
        """Abar = <A> - (1/|Omega|) L_f^T K_ff^-1 L_f  (the condensed form of Eq. k-mac-element-6)."""
        d = self.d
        Pm, Fm, Wm, Am = self.averages(w, Fbar)
        K = self.tangent(w, Fbar)
        Kff = K[self.free][:, self.free].tocsc()
        L = self.dR_dFbar(w, Fbar)[self.free]
        X = spla.splu(Kff).solve(L)
        Abar = Am.reshape(d * d, d * d) - (L.T @ X) / self.volume
        return Abar.reshape(d, d, d, d)

    def solve(self, Fbar, w0=None, rtol=1e-10, atol=1e-14, max_iter=30, max_steps=None, tangent=True, stages=1):
        """Full RVE solve: Newton, then Pbar, Wbar, <F> and (optionally) Abar.

        stages > 1: load continuation from w = 0 (w0 is ignored); Newton solves at
        I + (k/stages)(Fbar - I), k = 1 .. stages, each starting from the previous solution."""
        Fbar = np.asarray(Fbar, dtype=np.float64)
        if stages > 1:
            I = np.eye(self.d)
            w0 = np.zeros(self.n_dof)
            for k in range(1, stages):
                w0, status, _, hist = self.newton(I + (k / stages) * (Fbar - I), w0, rtol, atol, max_iter, max_steps)
                if status not in (STATUS_OK, STATUS_NEWTON_CAP):
                    return {"w": w0, "status": status, "newton_iters": 0, "history": hist}
        w, status, it, hist = self.newton(Fbar, w0, rtol, atol, max_iter, max_steps)
        out = {"w": w, "status": status, "newton_iters": it, "history": hist}
        if status in (STATUS_OK, STATUS_NEWTON_CAP):
            P, Fm, W, _ = self.averages(w, Fbar)
            out.update(P=P, F_mean=Fm, W=W)
            if tangent:
                out["A"] = self.condensed_tangent(w, Fbar)
        return out

    # ---------------------------------------------- paper's literal stiffness transfer
    def stiffness_transfer_T(self, w, Fbar, gradN, Nval, omega=1.0):
        """k^H = omega/|K_delta| T^T K^h_T T (Eq. k-mac-element-6/7).

        Column (I, i) of T is the micro displacement that solves the saddle-point system
        ch_3_eq_30 on the NON-periodic (n+1)^d node grid, driven by the linearised macro unit
        state u = N_I(x_K) e_i + (X - X_c) . grad N_I(x_K) e_i (Eq. linearization-uH), with G
        holding the non-redundant periodic partner constraints plus one pinned node.
        gradN: (N_node, d) macro shape-function gradients at the qp; Nval: (N_node,) values."""
        d, n = self.d, self.n
        ke, _ = self.element_tangents(w, Fbar)
        nn = (n + 1) ** d
        K = self._assemble(ke, self.conn_np, nn)  # full stiffness on the non-periodic grid
        ijk = np.array(list(itertools.product(range(n + 1), repeat=d)))[:, ::-1]
        X = ijk / n
        # constraint rows: every node with some index == n is tied to its periodic image
        rows = []
        dep = np.nonzero((ijk == n).any(axis=1))[0]
        img = ((ijk[dep] % n) * (n + 1) ** np.arange(d)).sum(-1)
        for p, q in zip(dep, img):
            for i in range(d):
                rows.append(((p * d + i, 1.0), (q * d + i, -1.0)))
        for i in range(d):  # pin node 0 (translation)
            rows.append(((i, 1.0),))
        m = len(rows)
        r_idx, c_idx, vals = [], [], []
        for r, entries in enumerate(rows):
            for c, v in entries:
                r_idx.append(r)
                c_idx.append(c)
                vals.append(v)
        Gm = sp.csr_matrix((vals, (r_idx, c_idx)), shape=(m, nn * d))
        KKT = sp.bmat([[K, Gm.T], [Gm, None]]).tocsc()
        lu = spla.splu(KKT)
        Xc = np.full(d, 0.5)
        N_node = gradN.shape[0]
        T = np.zeros((nn * d, N_node * d))
        for I in range(N_node):
            for i in range(d):
                dbar = np.zeros((nn, d))
                dbar[:, i] = Nval[I] + (X - Xc) @ gradN[I]
                rhs = np.concatenate([np.zeros(nn * d), Gm @ dbar.reshape(-1)])
                T[:, I * d + i] = lu.solve(rhs)[: nn * d]
        return omega / self.volume * (T.T @ (K @ T))
