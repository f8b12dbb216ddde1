"""Macro FE-HMM problem in FP64 (oracle; test infrastructure only).

Sec. 3.1 of the paper: the macro displacement is interpolated with standard
shape functions (Eq. u^H,u^h); at each macro quadrature point the RVE is driven
by the linearised macro field (Eq. linearization-uH), whose gradient gives
Fbar = I + Grad u^H.  The internal force is f_I = int B_I^T S^H (Eq. f_I^int)
with S^H = <F>^-1 <P> (Eq. macro-mean-stress); because P : Grad dv = S : dE this
equals sum_qp omega Pbar Grad N_I, which is what is assembled here (the tests
check the S^H route gives the same vector).  The tangent replaces the unknown
macro law by the RVE-averaged one (Eq. ModifiedBilinearForm-1/3), assembled as
k_IJ = sum_qp omega Grad N_I . Abar . Grad N_J (Eq. Assem_k_T_IK_mac with the
condensed Abar; equality with the T-matrix form of Eq. k-mac-element-6 is
checked in the tests).  omega = Gauss weight x det J.

The paper uses P1 triangles on the macro scale; the workloads here use Q1 (2D)
and Hex8 (3D) on the unit square/cube with 2^d Gauss points.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .rve import corner_offsets, gauss_points, shape_and_grad


class MacroMesh:
    def __init__(self, macro_n):
        self.n = tuple(int(m) for m in macro_n)
        d = self.d = len(self.n)
        h = 1.0 / np.array(self.n, dtype=np.float64)
        idx = np.array(list(itertools.product(*[range(m) for m in self.n[::-1]])))[:, ::-1]
        strides = np.cumprod([1] + [m + 1 for m in self.n[:-1]])
        off = corner_offsets(d)
        self.conn = ((idx[:, None, :] + off[None, :, :]) * strides).sum(-1)
        nidx = np.array(list(itertools.product(*[range(m + 1) for m in self.n[::-1]])))[:, ::-1]
        self.X = nidx * h
        self.n_nodes = self.X.shape[0]
        self.n_dof = self.n_nodes * d
        self.n_el = idx.shape[0]
        xi = gauss_points(d)
        self.Nq, self.G = shape_and_grad(d, xi, h)
        self.nq = xi.shape[0]
        self.n_qp = self.n_el * self.nq
        self.omega = float(np.prod(h / 2.0))  # Gauss weight 1 times det J, same for every qp
        self.x_qp = np.einsum("qa,ead->eqd", self.Nq, self.X[self.conn]).reshape(-1, d)

    def qp_F(self, u):
        """Fbar = I + sum_I u_I (x) Grad N_I at every macro qp: (n_qp, d, d)."""
        ue = u.reshape(self.n_nodes, self.d)[self.conn]
        F = np.eye(self.d)[None, None] + np.einsum("eai,qaJ->eqiJ", ue, self.G)
        return F.reshape(self.n_qp, self.d, self.d)

    def assemble(self, P, A):
        """f_I = sum omega Pbar Grad N_I and K_IJ = sum omega Grad N_I . Abar . Grad N_J."""
        d, nq = self.d, self.nq
        Pe = P.reshape(self.n_el, nq, d, d)
        Ae = A.reshape(self.n_el, nq, d, d, d, d)
        fe = self.omega * np.einsum("eqiJ,qaJ->eai", Pe, self.G)
        f = np.zeros((self.n_nodes, d))
        np.add.at(f, self.conn, fe)
        ke = self.omega * np.einsum("qaJ,eqiJkL,qbL->eaibk", self.G, Ae, self.G)
        nen = self.G.shape[1]
        dofs = (self.conn[:, :, None] * d + np.arange(d)[None, None, :]).reshape(self.n_el, -1)
        rows = np.repeat(dofs, nen * d, axis=1).reshape(-1)
        cols = np.tile(dofs, (1, nen * d)).reshape(-1)
        K = sp.csr_matrix((ke.reshape(-1), (rows, cols)), shape=(self.n_dof, self.n_dof))
        return f.reshape(-1), K

    def assemble_f_via_S(self, P, F):
        """f_I = int B_I^T S^H with S^H = <F>^-1 <P> (Eq. f_I^int, Eq. macro-mean-stress), using
        the Green-Lagrange variation dE = sym(F^T Grad dv) written out per component."""
        d, nq = self.d, self.nq
        S = np.linalg.solve(F, P)  # <F>^-1 <P>
        Se = S.reshape(self.n_el, nq, d, d)
        Fe = F.reshape(self.n_el, nq, d, d)
        # dE_IJ / d(u_a,i) = 1/2 (F_iI N_a,J + F_iJ N_a,I); S : dE
        fe = self.omega * 0.5 * (np.einsum("eqIJ,eqiI,qaJ->eai", Se, Fe, self.G)
                                 + np.einsum("eqIJ,eqiJ,qaI->eai", Se, Fe, self.G))
        f = np.zeros((self.n_nodes, d))
        np.add.at(f, self.conn, fe)
        return f.reshape(-1)

    def solve_increment(self, K, f, dirichlet_dofs):
        """Newton correction du with du = 0 on Dirichlet dofs: K_ff du_f = -f_f."""
        free = np.setdiff1d(np.arange(self.n_dof), dirichlet_dofs)
        du = np.zeros(self.n_dof)
        du[free] = spla.spsolve(K[free][:, free].tocsc(), -f[free])
        return du, free
