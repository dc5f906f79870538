"""PAW finite-element operators for the oracle (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

H = H_loc + sum_a P^a Delta_H^a P^a^T        (Eq. FE nonlocal contribution)
S = M     + sum_a P^a Delta_S^a P^a^T
H_loc = 1/2 K + V_mass                        (Eq. hij / FEM Ham entries, k = 0)

S^-1 exact: Woodbury over all atoms jointly on the consistent mass M.
S^-1 approx (Eqs. Sinvapprox, Delta Sinv):
    Shat^-1 = M_D^-1 - sum_a M_D^-1 P^a Dsinv^a P^a^T M_D^-1,
    Dsinv^a = (Delta_S^a^-1 + P^a^T M_D^-1 P^a)^-1
            = Delta_S^a (I + G_a Delta_S^a)^-1,   G_a = P^a^T M_D^-1 P^a
(the second form needs no inverse of Delta_S, which may be singular).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe


class PawOperators:
    """All operators of one workload, built from its seeded description.

    ``Vq`` overrides the potential at the (p+2)^3 quadrature points
    (shape (ncells, nq)); ``D`` / ``dS`` override the coupling matrices.
    """

    def __init__(self, sysd: dict, Vq=None, D=None, dS=None, pp_overlap=False):
        self.sysd = sysd
        self.mesh = m = fe.Mesh(sysd["L"], sysd["ncell"], sysd["p"])
        self.K = fe.kinetic_cell(m)
        self.Me = fe.mass_cell(m)
        self.Nq, _ = fe.basis3d(m, m.p + 2)
        self.Wq = fe.vquad_weights(m)
        self.Vq = fe.potential_at_quad(m, sysd) if Vq is None else np.asarray(Vq, float)
        self.md = fe.lumped_mass(m)
        self.D = np.asarray(sysd["D"] if D is None else D, float)
        self.dS = np.asarray(sysd["dS"] if dS is None else dS, float)
        self.natoms = int(sysd["natoms"])
        self.npj = int(sysd["nproj"])
        self.P = [fe.projector_matrix(m, sysd, a) for a in range(self.natoms)]
        # assembly operator Q: cell arrays (ncells*nc) -> global DoFs
        rows = m.cell_dofs.reshape(-1)
        cols = np.arange(rows.size)
        self.Q = sp.csr_matrix((np.ones(rows.size), (rows, cols)),
                               shape=(m.ndof, rows.size))
        # G_a and Dsinv_a (Eq. Delta Sinv)
        self.G = []
        self.Dsinv = []
        Gpp = fe.projector_overlap_analytic(sysd["shells"]) if pp_overlap else None
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            Ga = Pv.T @ (Pv / self.md[dofs, None]) if Gpp is None else Gpp
            self.G.append(Ga)
            I = np.eye(self.npj)
            self.Dsinv.append(self.dS[a] @ np.linalg.inv(I + Ga @ self.dS[a]))
        self._Minv = None
        self._Sinv_small = None

    # ---------------------------------------------------------------- helpers
    def _gather(self, X):
        return X[self.mesh.cell_dofs]                      # (ncells, nc, ncols)

    def _assemble(self, Ye):
        return self.Q @ Ye.reshape(-1, Ye.shape[-1])

    def _nonlocal(self, X, coup):
        Y = np.zeros_like(X)
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            U = Pv.T @ X[dofs]                             # P^a^T X
            Y[dofs] += Pv @ (coup[a] @ U)
        return Y

    # ---------------------------------------------------------------- H, S
    def apply_Hloc(self, X):
        """(1/2 K + V_mass) X by cell gather, cell product and assembly."""
        X = np.asarray(X, float)
        Xe = self._gather(X)
        Ye = np.matmul(self.K, Xe)                         # (1/2) K^e X_e, every cell
        U = np.matmul(self.Nq, Xe)                         # values at quad points
        U *= (self.Wq[None, :] * self.Vq)[:, :, None]
        Ye += np.matmul(self.Nq.T, U)                      # + V^e X_e
        return self._assemble(Ye)

    def apply_H(self, X):
        X = np.asarray(X, float)
        return self.apply_Hloc(X) + self._nonlocal(X, self.D)

    def apply_M(self, X):
        X = np.asarray(X, float)
        Ye = np.matmul(self.Me, self._gather(X))
        return self._assemble(Ye)

    def apply_S(self, X):
        X = np.asarray(X, float)
        return self.apply_M(X) + self._nonlocal(X, self.dS)

    # ---------------------------------------------------------------- S^-1
    def apply_Sinv_approx(self, X):
        """Shat^-1 X per Eqs. Sinvapprox / Delta Sinv (per-atom, lumped M_D)."""
        X = np.asarray(X, float)
        Z = X / self.md[:, None]
        corr = np.zeros_like(X)
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            corr[dofs] += Pv @ (self.Dsinv[a] @ (Pv.T @ Z[dofs]))
        return Z - corr / self.md[:, None]

    def _mass_solve(self, B):
        if self._Minv is None:
            Mglob = self.assembled_mass()
            self._Minv = spla.splu(Mglob.tocsc())
        return self._Minv.solve(np.asarray(B, float))

    def apply_Sinv_exact(self, X):
        """Exact S^-1 X by Woodbury over all atoms, consistent mass M."""
        X = np.asarray(X, float)
        Pall = self.projector_block()                      # (ndof, natoms*npj) sparse
        if self._Sinv_small is None:
            MP = self._mass_solve(Pall.toarray())
            Gall = Pall.T @ MP
            DS = sla.block_diag(*self.dS)
            self._Sinv_small = (MP, DS @ np.linalg.inv(np.eye(DS.shape[0]) + Gall @ DS))
        MP, core = self._Sinv_small
        Y = self._mass_solve(X)
        return Y - MP @ (core @ (Pall.T @ Y))

    # ---------------------------------------------------------------- assembled
    def projector_block(self):
        if self.natoms == 0:
            return sp.csr_matrix((self.mesh.ndof, 0))
        rows, cols, vals = [], [], []
        for a in range(self.natoms):
            dofs, Pv = self.P[a]
            r, c = np.meshgrid(dofs, np.arange(self.npj) + a * self.npj, indexing="ij")
            rows.append(r.ravel())
            cols.append(c.ravel())
            vals.append(Pv.ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.mesh.ndof, self.natoms * self.npj))

    def _assemble_cells(self, cellmats):
        m = self.mesh
        nc = m.nc
        rows = np.repeat(m.cell_dofs, nc, axis=1).reshape(-1)
        cols = np.tile(m.cell_dofs, (1, nc)).reshape(-1)
        return sp.csr_matrix((cellmats.reshape(-1), (rows, cols)), shape=(m.ndof, m.ndof))

    def assembled_mass(self):
        m = self.mesh
        return self._assemble_cells(np.broadcast_to(self.Me, (m.ncells, m.nc, m.nc)).copy())

    def cell_hamiltonians(self):
        """H^e = 1/2 K + V^e for every cell (ncells, nc, nc)."""
        out = np.empty((self.mesh.ncells, self.mesh.nc, self.mesh.nc))
        for e in range(self.mesh.ncells):
            out[e] = self.K + self.Nq.T @ ((self.Wq * self.Vq[e])[:, None] * self.Nq)
        return out

    def dense_H(self):
        Hl = self._assemble_cells(self.cell_hamiltonians()).toarray()
        if self.natoms == 0:
            return Hl
        Pall = self.projector_block().toarray()
        return Hl + Pall @ sla.block_diag(*self.D) @ Pall.T

    def dense_S(self):
        Ml = self.assembled_mass().toarray()
        if self.natoms == 0:
            return Ml
        Pall = self.projector_block().toarray()
        return Ml + Pall @ sla.block_diag(*self.dS) @ Pall.T
