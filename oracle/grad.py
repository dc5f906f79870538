"""Gradient of the subspace energy E = tr(X^T H X) (oracle, FP64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

H depends linearly on V (through V^e_IJ = sum_q w_q detJ V_q N_I N_J,
Eq. FEM Ham entries) and on the coupling matrices Delta_H^a (through
Eq. FE nonlocal contribution), so with X fixed:

  dE/dV_{e,q}          = w_q detJ sum_i u_i(x_q)^2,   u_i = sum_I N_I(x_q) X_{e,I,i}
  dE/dDelta_H^a[al,be] = sum_i U^a_{al,i} U^a_{be,i},  U^a = P^a^T X

Entries of Delta_H are treated as independent (the full n_pj x n_pj matrix;
the derivative with respect to a symmetric pair counts both entries).
"""
from __future__ import annotations

import numpy as np


def energy(ops, X) -> float:
    X = np.asarray(X, float)
    return float(np.sum(X * ops.apply_H(X)))


def energy_grad(ops, X):
    X = np.asarray(X, float)
    Xe = X[ops.mesh.cell_dofs]                                # (ncells, nc, n)
    U = np.einsum("qj,ejv->eqv", ops.Nq, Xe)
    dV = ops.Wq[None, :] * np.sum(U * U, axis=-1)
    dD = np.empty((ops.natoms, ops.npj, ops.npj))
    for a in range(ops.natoms):
        dofs, Pv = ops.P[a]
        Ua = Pv.T @ X[dofs]
        dD[a] = Ua @ Ua.T
    return dV, dD


def density(ops, X, occ=None):
    """Valence pseudo-density at the Gauss points and PAW occupation matrices.

    Eq. FE PAW governing equations at the Gamma point, one spin channel, without
    the core density and the compensation charges:
      rho(x_q) = sum_i f_i u_i(x_q)^2,          u_i = sum_I N_I(x_q) X_{e,I,i}
      D^a      = sum_i f_i U^a_i (U^a_i)^T,     U^a = P^a^T X
    Returns (rho as (ncells, nq), D as (natoms, npj, npj)).
    """
    X = np.asarray(X, float)
    f = np.ones(X.shape[1]) if occ is None else np.asarray(occ, float)
    Xe = X[ops.mesh.cell_dofs]                                # (ncells, nc, n)
    U = np.einsum("qj,ejv->eqv", ops.Nq, Xe)
    rho = np.einsum("eqv,v->eq", U * U, f)
    D = np.empty((ops.natoms, ops.npj, ops.npj))
    for a in range(ops.natoms):
        dofs, Pv = ops.P[a]
        Ua = Pv.T @ X[dofs]
        D[a] = (Ua * f) @ Ua.T
    return rho, D
