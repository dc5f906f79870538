"""Pins for the oracle's PAW operators (Eq. FE nonlocal contribution,
Eqs. Sinvapprox and Delta Sinv)."""
import numpy as np
import scipy.linalg as sla

from oracle import fe
from oracle import ops as O
from tests.oracle_systems import mini_system, sym_random


def _two_atom(separated=False, seed=3):
    rng = np.random.default_rng(seed)
    if separated:
        pos = [[6.1, 5.9, 6.2], [17.9, 18.2, 18.1]]
        shells = [(0, 0.3), (1, 0.3)]
        L, n, p = 24.0, 6, 3
    else:
        pos = [[2.1, 3.7, 4.9], [6.2, 5.1, 3.3]]
        shells = [(0, 0.8), (1, 0.8)]
        L, n, p = 10.0, 2, 4
    D = sym_random(rng, 2, 4, 0.1)
    dS = sym_random(rng, 2, 4, 0.02)
    return mini_system(L=L, n=n, p=p, positions=pos, shells=shells, D=D, dS=dS,
                       vdepth=2.0, vwidth=1.0)


def test_symmetry_and_spd():
    op = O.PawOperators(_two_atom())
    rng = np.random.default_rng(0)
    x = rng.standard_normal((op.mesh.ndof, 1))
    y = rng.standard_normal((op.mesh.ndof, 1))
    hxy = (x.T @ op.apply_H(y)).item()
    hyx = (y.T @ op.apply_H(x)).item()
    assert abs(hxy - hyx) < 1e-12 * max(1.0, abs(hxy))
    sxy = (x.T @ op.apply_S(y)).item()
    syx = (y.T @ op.apply_S(x)).item()
    assert abs(sxy - syx) < 1e-12 * max(1.0, abs(sxy))
    S = op.dense_S()
    np.linalg.cholesky(S)                       # S is SPD


def test_cell_form_matches_assembled():
    """apply_H (gather/cell product/assembly, quadrature-form V) == dense H."""
    op = O.PawOperators(_two_atom())
    X = np.random.default_rng(1).standard_normal((op.mesh.ndof, 3))
    H = op.dense_H()
    np.testing.assert_allclose(op.apply_H(X), H @ X, atol=1e-12 * np.abs(H).max())


def test_nonlocal_rank_and_sign():
    """H - H_loc = sum_a P^a D^a P^a^T: rank <= natoms*npj, spectrum of D."""
    s = _two_atom()
    op = O.PawOperators(s)
    dH = op.dense_H() - O.PawOperators(s, D=np.zeros_like(s["D"])).dense_H()
    ev = np.linalg.eigvalsh(dH)
    tiny = np.abs(ev) < 1e-10 * np.abs(ev).max()
    assert (~tiny).sum() == 8
    # with D = +I the nonlocal part is positive semidefinite
    I = np.broadcast_to(np.eye(4), s["D"].shape).copy()
    dI = O.PawOperators(s, D=I).dense_H() - O.PawOperators(s, D=0 * I).dense_H()
    assert np.linalg.eigvalsh(dI).min() > -1e-10


def test_exact_inverse():
    op = O.PawOperators(_two_atom())
    X = np.random.default_rng(2).standard_normal((op.mesh.ndof, 2))
    Y = op.apply_Sinv_exact(X)
    np.testing.assert_allclose(op.apply_S(Y), X, atol=1e-11)


def test_approx_inverse_exact_for_disjoint_atoms():
    """With node-disjoint supports Shat^-1 is the exact inverse of M_D + sum P dS P^T."""
    s = _two_atom(separated=True)
    op = O.PawOperators(s)
    d0, P0 = op.P[0]
    d1, P1 = op.P[1]
    nz0 = d0[np.abs(P0).max(1) > 0]
    nz1 = d1[np.abs(P1).max(1) > 0]
    assert len(nz0) > 0 and len(nz1) > 0 and len(np.intersect1d(nz0, nz1)) == 0
    X = np.random.default_rng(4).standard_normal((op.mesh.ndof, 2))
    Y = op.apply_Sinv_approx(X)
    SD = op.md[:, None] * Y
    for a in range(2):
        dofs, Pv = op.P[a]
        SD[dofs] += Pv @ (s["dS"][a] @ (Pv.T @ Y[dofs]))
    np.testing.assert_allclose(SD, X, atol=1e-11)


def test_approx_inverse_symmetric():
    op = O.PawOperators(_two_atom())
    rng = np.random.default_rng(5)
    x = rng.standard_normal((op.mesh.ndof, 1))
    y = rng.standard_normal((op.mesh.ndof, 1))
    a = (x.T @ op.apply_Sinv_approx(y)).item()
    b = (y.T @ op.apply_Sinv_approx(x)).item()
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))


def test_pp_overlap_option_close_to_exact_G():
    """<p|p> approximates C^T M_D^-1 C on a fine mesh (mesh-refinement limit)."""
    s = mini_system(L=8.0, n=4, p=6, positions=[[4.05, 3.9, 4.1]], shells=[(0, 0.8), (1, 0.8)])
    op = O.PawOperators(s)
    Gpp = fe.projector_overlap_analytic(s["shells"])
    np.testing.assert_allclose(op.G[0], Gpp, atol=5e-3)
