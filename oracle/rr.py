"""Rayleigh-Ritz, residuals, spectral bounds and the R-ChFSI driver (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Algorithm 1: bounds (generalised Lanczos) -> CF (Algorithm 2) ->
RR-Projection (H^p = Psi_f^T H Psi_f, S^p = Psi_f^T S Psi_f) ->
RR-GHEP (H^p Q = S^p Q Lambda) -> RR-SR (Psi = Psi_f Q).
Residual norms ||H psi_i - lambda_i S psi_i||_2 (Sec. 4, first paragraph).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import cheb


def rayleigh_ritz(ops, Xf):
    """Steps 4-6 of Algorithm 1 in FP64. Returns (Psi, lambda) ascending.

    H^p = Psi_f^dagger H Psi_f (the transpose for real blocks, the conjugate
    transpose for complex ones at a Bloch wavevector k).
    """
    HX = ops.apply_H(Xf)
    SX = ops.apply_S(Xf)
    Xh = Xf.conj().T
    Hp = Xh @ HX
    Sp = Xh @ SX
    Hp = 0.5 * (Hp + Hp.conj().T)
    Sp = 0.5 * (Sp + Sp.conj().T)
    lam, Q = sla.eigh(Hp, Sp)
    return Xf @ Q, lam


def residual_norms(ops, Psi, lam):
    """||H psi_i - lambda_i S psi_i||_2 per column (unweighted Euclidean)."""
    R = ops.apply_H(Psi) - ops.apply_S(Psi) * lam[None, :]
    return np.linalg.norm(R, axis=0)


def lanczos_bounds(apply_SinvH, apply_S, ndof: int, k: int = 20, seed: int = 7):
    """k-step generalised Lanczos on S^-1 H in the S inner product.

    Returns (theta_min, upper) where upper = theta_max + |beta_k s_k| is the
    usual safe bound on the largest eigenvalue.  The algorithm text of the
    paper's reference is not available; this is the textbook process.
    """
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(ndof)
    v = v / np.sqrt(np.vdot(v, apply_S(v[:, None])[:, 0]).real)
    vprev = np.zeros(ndof)
    alphas, betas = [], []
    beta = 0.0
    for _j in range(k):
        w = apply_SinvH(v[:, None])[:, 0]
        a = np.vdot(v, apply_S(w[:, None])[:, 0]).real      # S inner product (Hermitian: real)
        w = w - a * v - beta * vprev
        Sw = apply_S(w[:, None])[:, 0]
        beta = float(np.sqrt(max(np.vdot(w, Sw).real, 0.0)))
        alphas.append(a)
        betas.append(beta)
        vprev, v = v, w / beta
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    th, s = np.linalg.eigh(T)
    return float(th[0]), float(th[-1] + abs(betas[-1] * s[-1, -1]))


def dense_eigs(ops, nev: int):
    """Brute force: lowest nev eigenpairs of the assembled dense (H, S)."""
    H = ops.dense_H()
    S = ops.dense_S()
    lam, V = sla.eigh(H, S, subset_by_index=[0, nev - 1])
    return lam, V


def subspace_angles_S(S_apply, U, V):
    """Principal angles between span(U) and span(V) in the S inner product.

    Both bases are made S-orthonormal (Cholesky of their S-Gram matrices).
    The cosines are the singular values of U_o^T S V_o; the sines are the
    S-norms of the part of V_o that is S-orthogonal to span(U_o), i.e. the
    square roots of the eigenvalues of R^T S R with R = V_o - U_o (U_o^T S V_o).
    Angles below pi/4 are taken from the sines and the others from the cosines:
    arccos of a cosine near 1 resolves an angle t only to about eps / t, the
    sine keeps its relative accuracy (Knyazev and Argentati, SIAM J. Sci.
    Comput. 23 (2002)).  Returns min(dim U, dim V) angles in ascending order.
    Pinned by test_oracle_rr::test_subspace_angles_* (same span, S-orthogonal
    spans, constructed spans with known angles).
    """
    def orth(A):
        G = A.T @ S_apply(A)
        L = np.linalg.cholesky(0.5 * (G + G.T))
        return np.linalg.solve(L, A.T).T
    Uo, Vo = orth(U), orth(V)
    if Vo.shape[1] > Uo.shape[1]:
        Uo, Vo = Vo, Uo
    C = Uo.T @ S_apply(Vo)
    cos = np.sort(np.clip(np.linalg.svd(C, compute_uv=False), 0.0, 1.0))[::-1]   # ascending angles
    R = Vo - Uo @ C
    G = R.T @ S_apply(R)
    sin = np.sqrt(np.clip(np.sort(np.linalg.eigvalsh(0.5 * (G + G.T))), 0.0, 1.0))
    small = sin < np.sqrt(0.5)
    return np.where(small, np.arcsin(sin), np.arccos(cos))


def rchfsi(ops, X0, m: int, iters: int, nwanted: int, sinv="approx", history=None):
    """Algorithm 1 with Algorithm 2 as the CF step (FP64 oracle driver).

    Iteration 0 applies RR to the random block (reading of the start).  The
    bounds: b_U from 20-step Lanczos with exact S^-1, a_0 = min(lowest Ritz
    value, Lanczos theta_min), b_W = largest Ritz value of the block.
    """
    sinv_f = ops.apply_Sinv_approx if sinv == "approx" else ops.apply_Sinv_exact
    tmin, bU = lanczos_bounds(lambda x: ops.apply_Sinv_exact(ops.apply_H(x)),
                              ops.apply_S, ops.mesh.ndof)
    Psi, lam = rayleigh_ritz(ops, X0)
    for _it in range(iters):
        a0 = min(lam[0], tmin)
        bW = lam[-1]
        Xf = cheb.rchfsi_filter(ops.apply_H, ops.apply_S, sinv_f, Psi, lam, m, a0, bW, bU)
        Psi, lam = rayleigh_ritz(ops, Xf)
        if history is not None:
            r = residual_norms(ops, Psi[:, :nwanted], lam[:nwanted])
            history.append((lam.copy(), r))
    return Psi, lam, (tmin, bU)
