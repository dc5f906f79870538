"""Pins of the k-point oracle (oracle/kpoint.py) against what the mathematics fixes.

* the empty periodic box separates at any k: its 3D spectrum is the sum of three
  spectra of the 1D Bloch problem, assembled here independently (numpy Legendre
  roots, monomial Lagrange basis);
* H(k), S(k) are Hermitian; H(-k) = conj H(k) (time reversal);
* k = 0 gives the real operators of oracle.ops;
* translating an atom by a lattice vector changes C^{a,k} by the phase e^{-i k.L}
  and leaves H(k), S(k) unchanged;
* Shat^-1(k) S_D(k) = I for node-disjoint atom supports;
* the lowest levels of the empty box approach 1/2 |k + G|^2 on a fine mesh;
* R-ChFSI (Algorithm 2 with Shat^-1) converges to the dense eigensolve at k.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import inputs
from oracle import cheb, fe, kpoint, ops, rr

K_TINY = np.array([0.11, -0.07, 0.05])


def small_system(L=10.0, n=2, p=2, positions=((3.1, 4.2, 5.7),), shells=((0, 0.8), (1, 0.8)), seed=5):
    rng = np.random.default_rng(seed)
    npj = sum(2 * l + 1 for l, _ in shells)
    na = len(positions)

    def sym(s):
        A = rng.normal(0, s, (na, npj, npj))
        return 0.5 * (A + A.transpose(0, 2, 1))
    pos = np.asarray(positions, float)
    return dict(L=L, ncell=n, p=p, natoms=na, shells=list(shells), positions=pos, nproj=npj,
                D=sym(0.1), dS=sym(0.02), vloc_centers=pos.copy(), vloc_depth=np.full(na, 2.0),
                vloc_width=np.full(na, 1.0))


def _lagrange_1d(nodes, x):
    """values and derivatives of the Lagrange basis on nodes at points x (monomial form)."""
    n = len(nodes)
    V = np.vander(nodes, n, increasing=True)
    coef = np.linalg.inv(V)                   # column j: coefficients of l_j
    P = np.vander(x, n, increasing=True)
    dP = np.zeros_like(P)
    dP[:, 1:] = P[:, :-1] * np.arange(1, n)
    return P @ coef, dP @ coef


def bloch_1d_spectrum(L, n, p, kx):
    """Eigenvalues of (1/2 K1 + 1/2 kx^2 M1 - i kx C1) v = lam M1 v on a periodic 1D mesh."""
    # GLL nodes: endpoints and the roots of P_p'
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots()
    gll = np.sort(np.concatenate([[-1.0, 1.0], inner.real]))
    gq, gw = np.polynomial.legendre.leggauss(p + 1)
    phi, dphi = _lagrange_1d(gll, gq)
    h = L / n
    Ke = (2.0 / h) * (dphi.T @ (gw[:, None] * dphi))          # int l_i' l_j' dx
    Me = (h / 2.0) * (phi.T @ (gw[:, None] * phi))
    Ce = phi.T @ (gw[:, None] * dphi)                          # int l_i l_j' dx
    N1 = n * p
    K = np.zeros((N1, N1))
    M = np.zeros((N1, N1))
    C = np.zeros((N1, N1))
    for c in range(n):
        idx = (c * p + np.arange(p + 1)) % N1
        K[np.ix_(idx, idx)] += Ke
        M[np.ix_(idx, idx)] += Me
        C[np.ix_(idx, idx)] += Ce
    H = 0.5 * K + 0.5 * kx * kx * M - 1j * kx * C
    return sla.eigh(H, M, eigvals_only=True)


def test_empty_box_separates_at_k():
    sysd = small_system(L=7.0, n=2, p=3, positions=())
    sysd.update(natoms=0, positions=np.zeros((0, 3)), D=np.zeros((0, 4, 4)), dS=np.zeros((0, 4, 4)),
                vloc_centers=np.zeros((0, 3)), vloc_depth=np.zeros(0), vloc_width=np.zeros(0))
    k = np.array([0.31, -0.17, 0.08])
    op = kpoint.PawOperatorsK(sysd, k)
    lam3 = sla.eigh(op.dense_H(), op.dense_S(), eigvals_only=True)
    l1 = [bloch_1d_spectrum(7.0, 2, 3, kd) for kd in k]
    sums = np.sort(np.add.outer(np.add.outer(l1[0], l1[1]), l1[2]).ravel())
    assert np.max(np.abs(lam3 - sums)) < 1e-10 * max(1.0, np.max(np.abs(sums)))


def test_empty_box_continuum_limit():
    """lowest Bloch levels approach 1/2 |k + 2 pi n / L|^2 on a fine mesh."""
    L = 6.0
    k = np.array([0.2, 0.0, 0.0])
    sysd = small_system(L=L, n=3, p=5, positions=())
    sysd.update(natoms=0, positions=np.zeros((0, 3)), D=np.zeros((0, 4, 4)), dS=np.zeros((0, 4, 4)),
                vloc_centers=np.zeros((0, 3)), vloc_depth=np.zeros(0), vloc_width=np.zeros(0))
    op = kpoint.PawOperatorsK(sysd, k)
    lam, _ = op.dense_eigs(3)
    g = 2 * np.pi / L
    exact = sorted(0.5 * np.sum((k + g * np.array(n)) ** 2)
                   for n in itertools.product(range(-2, 3), repeat=3))[:3]
    assert np.max(np.abs(lam - np.array(exact))) < 1e-6


def test_hermitian_and_time_reversal():
    sysd = inputs.make_system("tiny")
    sysd = dict(sysd, ncell=2, p=3)
    op = kpoint.PawOperatorsK(sysd, K_TINY)
    H, S = op.dense_H(), op.dense_S()
    assert np.max(np.abs(H - H.conj().T)) < 1e-13 * np.max(np.abs(H))
    assert np.max(np.abs(S - S.conj().T)) < 1e-13 * np.max(np.abs(S))
    opm = kpoint.PawOperatorsK(sysd, -K_TINY)
    assert np.max(np.abs(opm.dense_H() - H.conj())) < 1e-13 * np.max(np.abs(H))
    assert np.max(np.abs(opm.dense_S() - S.conj())) < 1e-13 * np.max(np.abs(S))
    assert np.min(np.linalg.eigvalsh(S)) > 0


def test_bloch_term_assembles_antisymmetric():
    """sum over cells of int N_I dN_J/dx is antisymmetric on the periodic box."""
    m = fe.Mesh(7.0, 2, 3)
    B = kpoint.bloch_cell(m, np.array([0.3, -0.2, 0.1]))
    G = np.zeros((m.ndof, m.ndof))
    for e in range(m.ncells):
        idx = m.cell_dofs[e]
        G[np.ix_(idx, idx)] += B
    assert np.max(np.abs(G + G.T)) < 1e-13 * np.max(np.abs(G))


def test_k0_reduces_to_gamma_operators():
    sysd = inputs.make_system("tiny")
    opk = kpoint.PawOperatorsK(sysd, np.zeros(3))
    op = ops.PawOperators(sysd)
    X = inputs.start_columns("tiny", range(3))
    for fk, f in ((opk.apply_H, op.apply_H), (opk.apply_S, op.apply_S),
                  (opk.apply_Sinv_approx, op.apply_Sinv_approx)):
        a, b = fk(X), f(X)
        assert np.max(np.abs(a.imag)) < 1e-14 * np.max(np.abs(b))
        assert np.max(np.abs(a.real - b)) < 1e-13 * np.max(np.abs(b))


def test_lattice_translation_of_an_atom():
    sysd = small_system(n=2, p=3)
    k = np.array([0.2, 0.1, -0.15])
    op = kpoint.PawOperatorsK(sysd, k)
    moved = dict(sysd, positions=sysd["positions"] + np.array([[10.0, 0.0, -10.0]]))
    op2 = kpoint.PawOperatorsK(moved, k)
    d1, P1 = op.P[0]
    d2, P2 = op2.P[0]
    assert np.array_equal(d1, d2)
    ph = np.exp(-1j * (k @ np.array([10.0, 0.0, -10.0])))
    assert np.max(np.abs(P2 - ph * P1)) < 1e-12 * np.max(np.abs(P1))
    assert np.max(np.abs(op2.dense_H() - op.dense_H())) < 1e-12
    assert np.max(np.abs(op2.dense_S() - op.dense_S())) < 1e-12


def test_sinv_approx_exact_on_disjoint_supports():
    sysd = small_system(L=30.0, n=6, p=2, positions=((5.0, 5.0, 5.0), (20.0, 20.0, 20.0)))
    op = kpoint.PawOperatorsK(sysd, np.array([0.05, 0.12, -0.09]))
    s0, s1 = ({int(d) for d, row in zip(*op.P[a]) if np.any(row != 0)} for a in range(2))
    assert s0 and s1 and not (s0 & s1)
    SD = np.diag(op.md).astype(complex)
    for a in range(2):
        dofs, Pv = op.P[a]
        SD[np.ix_(dofs, dofs)] += Pv @ op.dS[a] @ Pv.conj().T
    X = np.random.default_rng(1).standard_normal((op.mesh.ndof, 3)) + 0j
    Y = op.apply_Sinv_approx(SD @ X)
    assert np.max(np.abs(Y - X)) < 1e-11


def test_rchfsi_converges_at_k():
    sysd = inputs.make_system("tiny")
    sysd = dict(sysd, ncell=3, p=3)
    op = kpoint.PawOperatorsK(sysd, K_TINY)
    exact, _ = op.dense_eigs(8)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((op.mesh.ndof, 12)) + 1j * rng.standard_normal((op.mesh.ndof, 12))
    tmin, bU = rr.lanczos_bounds(lambda x: op.apply_Sinv_exact(op.apply_H(x)), op.apply_S, op.mesh.ndof)
    Psi, lam = rr.rayleigh_ritz(op, X)
    for _ in range(10):
        Xf = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, 16,
                                min(lam[0], tmin), lam[-1], bU)
        Psi, lam = rr.rayleigh_ritz(op, Xf)
    assert np.max(np.abs(lam[:8] - exact)) < 1e-8
    assert bU >= np.max(sla.eigh(op.dense_H(), op.dense_S(), eigvals_only=True)) - 1e-8
