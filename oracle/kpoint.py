"""PAW finite-element operators at a Bloch wavevector k (FP64 complex, numpy/scipy).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Local part (Eq. hij, with the Gamma-point terms of ops.py):
    H_loc(k)_IJ = int [1/2 grad N_I . grad N_J + V N_I N_J + 1/2 |k|^2 N_I N_J
                       - i k . N_I grad N_J] dx
The kinetic, |k|^2 and k . grad terms use the (p+1)^3 Gauss rule (Sec. 4.1,
n_q1), the potential the (p+2)^3 rule.  The k . grad term is taken with the
sign of Eq. hij (the cell-level form, Eq. FEM Ham entries, prints the
transposed product; the two differ by a sign after assembly).  Eq. hij is the
weak form of 1/2 |(grad + i k) u|^2 for the periodic factor u of
psi = e^{i k.x} u, which is also the convention of the Bloch phases below.

Projectors with Bloch phases (Eqs. FE nonlocal contribution, FEM Cmatrix):
    C^{a,k}_{J alpha} = sum_r int e^{-i k.(x - L_r)} p_alpha(x - R_a - L_r) N_J(x) dx
with one periodic image per point (cut-off radius below L/2): x - L_r = R_a + d,
d the minimum-image displacement.

    H(k) = H_loc(k) + sum_a C^a Delta_H^a C^a^dagger
    S(k) = M + sum_a C^a Delta_S^a C^a^dagger
    Shat^-1(k) = M_D^-1 - sum_a M_D^-1 C^a Dsinv^a C^a^dagger M_D^-1,
    Dsinv^a = Delta_S^a (I + G_a Delta_S^a)^-1,  G_a = C^a^dagger M_D^-1 C^a
Pinned by tests/test_oracle_kpoint.py: the separable spectrum of the empty box
at k against an independently assembled 1D problem, Hermiticity, time reversal
H(-k) = conj H(k), the k = 0 reduction to ops.PawOperators, the phase
e^{-i k.L} of C^{a,k} under a lattice translation of an atom (H, S unchanged),
Shat^-1 exact on node-disjoint supports, the continuum limit 1/2 |k + G|^2 of
the empty box, and convergence of Algorithm 2 to the dense eigensolve.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe


def bloch_cell(mesh: fe.Mesh, k) -> np.ndarray:
    """B^e_IJ = sum_d k_d int_e N_I dN_J/dx_d dx ((p+1)^3 Gauss); real, equal for every cell.

    The local k . grad term of Eq. hij is -i B (assembled over cells).
    """
    N, G = fe.basis3d(mesh, mesh.p + 1)
    n1 = mesh.p + 1
    _, w = fe.gauss_rule(n1)
    qi = np.arange(n1 ** 3)
    W = w[qi % n1] * w[(qi // n1) % n1] * w[qi // (n1 * n1)]
    s = (2.0 / mesh.h) * mesh.detJ                        # d/dx = (2/h) d/dxi
    B = np.zeros((mesh.nc, mesh.nc))
    for d in range(3):
        B += k[d] * s * (N.T @ (W[:, None] * G[d]))
    return B


def projector_matrix_k(mesh: fe.Mesh, sysd: dict, atom: int, k):
    """Assembled C^{a,k} for one atom: (dofs, complex values (len(dofs), npj))."""
    shells = sysd["shells"]
    R = np.asarray(sysd["positions"][atom], float)
    rmax = max(fe.cutoff_radius(w) for _, w in shells)
    N, _ = fe.basis3d(mesh, mesh.p + 2)
    pts, W = mesh.quad_points(mesh.p + 2)
    centres = (mesh.cell_xyz + 0.5) * mesh.h
    dc = fe.min_image(centres - R, mesh.L)
    near = np.nonzero(np.linalg.norm(dc, axis=1) < rmax + mesh.h * math.sqrt(3) / 2 + 1e-12)[0]
    npj = sysd["nproj"]
    d = fe.min_image(pts[near] - R, mesh.L)               # (nnear, nq, 3)
    pv = fe.projector_values(shells, d)                   # (nnear, nq, npj)
    phase = np.exp(-1j * ((R[None, None, :] + d) @ np.asarray(k, float)))   # e^{-i k.(x - L_r)}
    Ce = np.matmul(N.T, ((W * mesh.detJ)[None, :] * phase)[:, :, None] * pv)
    alldofs = mesh.cell_dofs[near].reshape(-1)
    dofs, inv = np.unique(alldofs, return_inverse=True)
    vals = np.zeros((len(dofs), npj), complex)
    np.add.at(vals, inv, Ce.reshape(-1, npj))
    return dofs, vals


class PawOperatorsK:
    """All operators of one workload at the Bloch wavevector k (Cartesian, 1/bohr)."""

    def __init__(self, sysd: dict, k, Vq=None):
        self.sysd = sysd
        self.k = np.asarray(k, float)
        self.mesh = m = fe.Mesh(sysd["L"], sysd["ncell"], sysd["p"])
        self.Me = fe.mass_cell(m)
        self.Hk = (fe.kinetic_cell(m) + 0.5 * float(self.k @ self.k) * self.Me
                   - 1j * bloch_cell(m, self.k))          # cell matrix without the potential
        self.Nq, _ = fe.basis3d(m, m.p + 2)
        self.Wq = fe.vquad_weights(m)
        self.Vq = fe.potential_at_quad(m, sysd) if Vq is None else np.asarray(Vq, float)
        self.md = fe.lumped_mass(m)
        self.D = np.asarray(sysd["D"], float)
        self.dS = np.asarray(sysd["dS"], float)
        self.natoms = int(sysd["natoms"])
        self.npj = int(sysd["nproj"])
        self.P = [projector_matrix_k(m, sysd, a, self.k) for a in range(self.natoms)]
        rows = m.cell_dofs.reshape(-1)
        self.Q = sp.csr_matrix((np.ones(rows.size), (rows, np.arange(rows.size))),
                               shape=(m.ndof, rows.size))
        self.G, self.Dsinv = [], []
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            Ga = Pv.conj().T @ (Pv / self.md[dofs, None])
            self.G.append(Ga)
            self.Dsinv.append(self.dS[a] @ np.linalg.inv(np.eye(self.npj) + Ga @ self.dS[a]))
        self._Mlu = None

    # ---------------------------------------------------------------- helpers
    def _gather(self, X):
        return X[self.mesh.cell_dofs]

    def _assemble(self, Ye):
        return self.Q @ Ye.reshape(-1, Ye.shape[-1])

    def _nonlocal(self, X, coup):
        Y = np.zeros(X.shape, complex)
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            Y[dofs] += Pv @ (coup[a] @ (Pv.conj().T @ X[dofs]))
        return Y

    # ---------------------------------------------------------------- H, S
    def apply_Hloc(self, X):
        Xe = self._gather(np.asarray(X, complex))
        Ye = np.matmul(self.Hk, Xe)
        U = np.matmul(self.Nq, Xe)
        U *= (self.Wq[None, :] * self.Vq)[:, :, None]
        Ye += np.matmul(self.Nq.T, U)
        return self._assemble(Ye)

    def apply_H(self, X):
        X = np.asarray(X, complex)
        return self.apply_Hloc(X) + self._nonlocal(X, self.D)

    def apply_M(self, X):
        return self._assemble(np.matmul(self.Me, self._gather(np.asarray(X, complex))))

    def apply_S(self, X):
        X = np.asarray(X, complex)
        return self.apply_M(X) + self._nonlocal(X, self.dS)

    def apply_Sinv_approx(self, X):
        X = np.asarray(X, complex)
        Z = X / self.md[:, None]
        corr = np.zeros_like(Z)
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            corr[dofs] += Pv @ (self.Dsinv[a] @ (Pv.conj().T @ Z[dofs]))
        return Z - corr / self.md[:, None]

    def _mass_solve(self, B):
        if self._Mlu is None:
            m = self.mesh
            nc = m.nc
            r = np.repeat(m.cell_dofs, nc, axis=1).reshape(-1)
            c = np.tile(m.cell_dofs, (1, nc)).reshape(-1)
            Mg = sp.csr_matrix((np.broadcast_to(self.Me, (m.ncells, nc, nc)).reshape(-1), (r, c)),
                               shape=(m.ndof, m.ndof))
            self._Mlu = spla.splu(Mg.tocsc())
        B = np.asarray(B, complex)
        return self._Mlu.solve(B.real) + 1j * self._Mlu.solve(B.imag)

    def projector_block(self):
        m = self.mesh
        Pall = np.zeros((m.ndof, self.natoms * self.npj), complex)
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            Pall[dofs, a * self.npj:(a + 1) * self.npj] = Pv
        return Pall

    def apply_Sinv_exact(self, X):
        """Exact S(k)^-1 X by Woodbury over all atoms on the consistent mass."""
        X = np.asarray(X, complex)
        Pall = self.projector_block()
        MP = self._mass_solve(Pall)
        DS = sla.block_diag(*self.dS)
        core = DS @ np.linalg.inv(np.eye(DS.shape[0]) + Pall.conj().T @ MP @ DS)
        Y = self._mass_solve(X)
        return Y - MP @ (core @ (Pall.conj().T @ Y))

    # ---------------------------------------------------------------- dense
    def dense_Hloc(self):
        m = self.mesh
        n = m.ndof
        H = np.zeros((n, n), complex)
        for e in range(m.ncells):
            He = self.Hk + self.Nq.T @ ((self.Wq * self.Vq[e])[:, None] * self.Nq)
            idx = m.cell_dofs[e]
            H[np.ix_(idx, idx)] += He
        return H

    def dense_H(self):
        H = self.dense_Hloc()
        if self.natoms:
            Pall = self.projector_block()
            H += Pall @ sla.block_diag(*self.D) @ Pall.conj().T
        return H

    def dense_S(self):
        m = self.mesh
        S = np.zeros((m.ndof, m.ndof), complex)
        for e in range(m.ncells):
            idx = m.cell_dofs[e]
            S[np.ix_(idx, idx)] += self.Me
        if self.natoms:
            Pall = self.projector_block()
            S += Pall @ sla.block_diag(*self.dS) @ Pall.conj().T
        return S

    def dense_eigs(self, nev: int):
        lam, V = sla.eigh(self.dense_H(), self.dense_S(), subset_by_index=[0, nev - 1])
        return lam, V
