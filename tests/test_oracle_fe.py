"""Pins for the oracle's finite-element discretisation (Sec. 2.2, Sec. 4.1).

Every check compares the oracle with something it does not compute itself:
textbook quadrature values, exactness of polynomial integration, the
separable spectrum of the empty periodic box, analytic Gaussian integrals.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from numpy.polynomial import legendre as npleg

from oracle import fe
from oracle import ops as O
from tests.oracle_systems import mini_system

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(s):
    return float(eval(s, {"sqrt": math.sqrt}))


def test_gll_textbook():
    g = json.load(open(os.path.join(GOLDEN, "gll_textbook.json")))
    for p, rule in g["rules"].items():
        x, w = fe.gll_rule(int(p))
        np.testing.assert_allclose(x, [_frac(s) for s in rule["nodes"]], atol=1e-14)
        np.testing.assert_allclose(w, [_frac(s) for s in rule["weights"]], atol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
def test_gll_exactness(p):
    x, w = fe.gll_rule(p)
    for k in range(2 * p):                      # exact up to degree 2p-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    # and not exact at degree 2p (so it is GLL, not Gauss)
    assert abs(np.sum(w * x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("p", [2, 4, 6])
def test_lagrange_properties(p):
    xi, _ = fe.gll_rule(p)
    phi, dphi = fe.lagrange(xi, xi)
    np.testing.assert_allclose(phi, np.eye(p + 1), atol=1e-14)
    t = np.linspace(-1, 1, 37)
    phi, dphi = fe.lagrange(xi, t)
    np.testing.assert_allclose(phi.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(dphi.sum(1), 0.0, atol=1e-11)
    # the interpolant of x^p is exact; so is its derivative
    np.testing.assert_allclose(phi @ xi ** p, t ** p, atol=1e-13)
    np.testing.assert_allclose(dphi @ xi ** p, p * t ** (p - 1), atol=1e-11)


def _periodic_1d(L, n, p):
    """1D periodic GHEP assembled in the test from 1D Lagrange elements."""
    xi, _ = fe.gll_rule(p)
    g, w = npleg.leggauss(p + 1)
    phi, dphi = fe.lagrange(xi, g)
    h = L / n
    Ke = (2.0 / h) * (dphi.T @ (w[:, None] * dphi))
    Me = (h / 2.0) * (phi.T @ (w[:, None] * phi))
    N = n * p
    K = np.zeros((N, N))
    M = np.zeros((N, N))
    for c in range(n):
        idx = [(c * p + a) % N for a in range(p + 1)]
        K[np.ix_(idx, idx)] += Ke
        M[np.ix_(idx, idx)] += Me
    return K, M


@pytest.mark.parametrize("L,n,p", [(10.0, 2, 3), (6.0, 3, 2), (5.0, 2, 4)])
def test_empty_box_separable(L, n, p):
    """Affine cubes with exact Gauss mass: 3D spectrum = sums of 1D spectra."""
    s = mini_system(L=L, n=n, p=p)
    op = O.PawOperators(s)
    H = op.dense_H()
    S = op.dense_S()
    lam3 = np.sort(sla.eigh(H, S, eigvals_only=True))
    K1, M1 = _periodic_1d(L, n, p)
    l1 = sla.eigh(0.5 * K1, M1, eigvals_only=True)
    sums = np.sort((l1[:, None, None] + l1[None, :, None] + l1[None, None, :]).ravel())
    np.testing.assert_allclose(lam3, sums, atol=1e-10 * max(1.0, sums.max()))


def test_empty_box_continuum_limit():
    """Lowest nonzero levels approach (1/2)(2 pi / L)^2 |n|^2 (6-fold degenerate)."""
    L = 10.0
    s = mini_system(L=L, n=3, p=5)
    op = O.PawOperators(s)
    lam = np.sort(sla.eigh(op.dense_H(), op.dense_S(), eigvals_only=True))
    k2 = 0.5 * (2 * math.pi / L) ** 2
    assert abs(lam[0]) < 1e-10
    np.testing.assert_allclose(lam[1:7], k2, rtol=1e-6)
    np.testing.assert_allclose(lam[7:19], 2 * k2, rtol=1e-5)


def test_kinetic_nullspace_and_mass_total():
    m = fe.Mesh(7.0, 2, 4)
    K = fe.kinetic_cell(m)
    Me = fe.mass_cell(m)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    np.testing.assert_allclose(K.sum(1), 0.0, atol=1e-12)
    assert np.linalg.eigvalsh(K).min() > -1e-12
    assert abs(Me.sum() - m.h ** 3) < 1e-12 * m.h ** 3
    assert np.linalg.eigvalsh(Me).min() > 0


def test_lumped_mass_total():
    m = fe.Mesh(9.0, 3, 5)
    md = fe.lumped_mass(m)
    assert md.min() > 0
    assert abs(md.sum() - m.L ** 3) < 1e-10 * m.L ** 3


def test_constant_potential_shift():
    """V = v0 everywhere adds v0 M to H, so every eigenvalue moves by v0."""
    s = mini_system(L=6.0, n=2, p=3)
    op0 = O.PawOperators(s)
    v0 = -0.731
    opv = O.PawOperators(s, Vq=np.full_like(op0.Vq, v0))
    l0 = np.sort(sla.eigh(op0.dense_H(), op0.dense_S(), eigvals_only=True))
    lv = np.sort(sla.eigh(opv.dense_H(), opv.dense_S(), eigvals_only=True))
    np.testing.assert_allclose(lv - l0, v0, atol=1e-10)


def test_linear_potential_exact():
    """V(x) = x: V^e equals the exact integral computed by 1D factorisation."""
    m = fe.Mesh(6.0, 2, 3)
    e = 5
    pts, _ = m.quad_points(m.p + 2)
    Ve = fe.potential_cell(m, pts[e, :, 0])
    # exact: int N_I N_J x = (int phi_a phi_a' x)(int phi_b phi_b')(int phi_c phi_c')
    g, w = npleg.leggauss(12)
    phi, _ = fe.lagrange(m.xi, g)
    x0 = m.cell_xyz[e, 0] * m.h
    xs = x0 + (g + 1) * m.h / 2
    Ax = (m.h / 2) * phi.T @ ((w * xs)[:, None] * phi)
    A1 = (m.h / 2) * phi.T @ (w[:, None] * phi)
    a, b, c = m.local_abc.T
    ref = Ax[np.ix_(a, a)] * A1[np.ix_(b, b)] * A1[np.ix_(c, c)]
    np.testing.assert_allclose(Ve, ref, atol=1e-13)


def test_projector_norm_and_overlap():
    """Brute-force integration on a fine grid: <p_a|p_b> matches the analytic form."""
    shells = [(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)]
    h = 0.09
    t = np.arange(-8.0, 8.0 + 1e-9, h)
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    d = np.stack([X, Y, Z], -1)
    pv = fe.projector_values(shells, d).reshape(-1, 13)
    G = (pv.T @ pv) * h ** 3
    Ga = fe.projector_overlap_analytic(shells)
    np.testing.assert_allclose(np.diag(G)[[0, 2, 3, 4, 8]], 1.0, atol=2e-4)
    np.testing.assert_allclose(G, Ga, atol=2e-3)


def test_projector_integral_moments():
    """Sum_J f(x_J) P^a_J = int f p for f in the FE space (1, x, xy)."""
    L = 12.0
    shells = [(0, 0.7), (1, 0.7), (2, 0.7)]
    s = mini_system(L=L, n=8, p=5, positions=[[6.1, 5.8, 6.3]], shells=shells)
    m = fe.Mesh(L, 8, 5)
    dofs, Pv = fe.projector_matrix(m, s, 0)
    x = fe.min_image(m.node_coords()[dofs] - s["positions"][0], L)
    w = 0.7
    gauss = (2 * math.pi * w * w) ** 1.5
    c00 = fe.radial_norm(0, w) * 0.5 / math.sqrt(math.pi)
    c1 = fe.radial_norm(1, w) * math.sqrt(3 / (4 * math.pi))
    c2 = fe.radial_norm(2, w) * 0.5 * math.sqrt(15 / math.pi)
    np.testing.assert_allclose(Pv[:, 0].sum(), c00 * gauss, rtol=1e-6)
    # l = 1 ordering m = -1, 0, 1  <->  y, z, x
    np.testing.assert_allclose(Pv[:, 1] @ x[:, 1], c1 * w * w * gauss, rtol=1e-6)
    np.testing.assert_allclose(Pv[:, 2] @ x[:, 2], c1 * w * w * gauss, rtol=1e-6)
    np.testing.assert_allclose(Pv[:, 3] @ x[:, 0], c1 * w * w * gauss, rtol=1e-6)
    assert abs(Pv[:, 3] @ x[:, 1]) < 1e-8
    # l = 2, m = -2 is xy (truncation at 6.07 w weighs more on r^4 moments)
    np.testing.assert_allclose(Pv[:, 4] @ (x[:, 0] * x[:, 1]), c2 * w ** 4 * gauss, rtol=3e-5)


def test_mesh_dof_map():
    m = fe.Mesh(5.0, 3, 2)
    # every DoF is reached, corners by 8 cells, interior nodes by 1
    counts = np.bincount(m.cell_dofs.ravel(), minlength=m.ndof)
    assert counts.min() >= 1 and counts.max() == 8
    assert counts.sum() == m.ncells * m.nc
    # node coordinates of a cell's local nodes lie in the cell (periodic)
    xyz = m.node_coords()
    e = 7
    loc = xyz[m.cell_dofs[e]]
    org = m.cell_xyz[e] * m.h
    rel = np.mod(loc - org + 1e-12, m.L) - 1e-12
    assert rel.min() >= -1e-12 and rel.max() <= m.h + 1e-12


# ---------------------------------------------------------------------------
# Synthetic local potential (reading of the configs: V = -sum A exp(-r^2 / (2 w^2))
# over periodic images within 8 w).  Pinned by values fixed by that definition and by
# the Poisson-summation closed form of the fully periodic Gaussian, which the oracle
# does not compute: sum_n exp(-(x - n L)^2 / (2 w^2))
#   = (w sqrt(2 pi) / L) [1 + 2 sum_{k>=1} exp(-2 pi^2 k^2 w^2 / L^2) cos(2 pi k x / L)].
# ---------------------------------------------------------------------------
def _theta_periodic(x, L, w, kmax=200):
    k = np.arange(1, kmax + 1)
    terms = np.exp(-2.0 * math.pi ** 2 * (k * w / L) ** 2)[None, :] * np.cos(2.0 * math.pi * np.outer(x, k) / L)
    return (w * math.sqrt(2.0 * math.pi) / L) * (1.0 + 2.0 * terms.sum(1))


def _poisson_potential(pts, L, centers, depth, width):
    V = np.zeros(len(pts))
    for R, A, w in zip(centers, depth, width):
        d = pts - np.asarray(R)
        V -= A * _theta_periodic(d[:, 0], L, w) * _theta_periodic(d[:, 1], L, w) * _theta_periodic(d[:, 2], L, w)
    return V


def test_gaussian_potential_values():
    """V at the centre is -A, at distance w it is -A e^{-1/2} (w is the standard deviation,
    not the 1/e radius), at 7.9 w it is -A e^{-7.9^2/2}, and beyond the 8 w image cut it is 0;
    the minimum image wraps across the box."""
    L, A, w = 40.0, 2.0, 1.0
    R = np.array([3.0, 20.0, 17.5])
    ex = np.array([1.0, 0.0, 0.0])
    pts = np.array([R, R + w * ex, R + 7.9 * w * ex, R + 8.1 * w * ex, R - w * ex + [L, 0.0, 0.0],
                    R + [0.0, L - w, 0.0], R + [0.0, 0.0, L]])
    V = fe.gaussian_potential(pts, L, [R], [A], [w])
    np.testing.assert_allclose(V[0], -A, rtol=1e-15)
    np.testing.assert_allclose(V[1], -A * math.exp(-0.5), rtol=1e-14)
    np.testing.assert_allclose(V[2], -A * math.exp(-7.9 ** 2 / 2), rtol=1e-12)
    assert V[3] == 0.0
    np.testing.assert_allclose(V[4:6], -A * math.exp(-0.5), rtol=1e-14)   # wrap by L, and by L - w
    np.testing.assert_allclose(V[6], -A, rtol=1e-15)                        # a lattice translate of the centre
    # superposition of two centres with their own depth and width
    R2, A2, w2 = np.array([5.0, 21.0, 17.5]), 1.5, 0.7
    V2 = fe.gaussian_potential(pts[:2], L, [R, R2], [A, A2], [w, w2])
    d2 = np.sum((pts[:2] - R2) ** 2, 1)
    np.testing.assert_allclose(V2, V[:2] - A2 * np.exp(-d2 / (2 * w2 * w2)), rtol=1e-14)


@pytest.mark.parametrize("L,cut", [(3.0, 12.0), (4.5, 12.0)])
def test_gaussian_potential_images_poisson(L, cut):
    """Image-sum branch (cut radius above L/2): with a cut far out in the tail the oracle's
    sum over periodic images equals the Poisson-summed closed form."""
    rng = np.random.default_rng(5)
    centers = rng.uniform(0, L, (2, 3))
    depth, width = [2.0, 1.3], [1.0, 0.8]
    assert cut * min(width) >= L / 2
    pts = rng.uniform(0, L, (40, 3))
    V = fe.gaussian_potential(pts, L, centers, depth, width, image_cut=cut)
    ref = _poisson_potential(pts, L, centers, depth, width)
    np.testing.assert_allclose(V, ref, rtol=1e-12, atol=0)


def test_gaussian_potential_minimum_image_poisson():
    """Minimum-image branch (the configs' boxes): the 8 w cut drops only the tail beyond 8 w,
    below A e^{-32}, so V agrees with the full periodic sum to 1e-12 A everywhere."""
    L = 40.0
    rng = np.random.default_rng(6)
    centers = rng.uniform(0, L, (3, 3))
    depth, width = [2.0, 2.0, 1.0], [1.0, 0.9, 1.2]
    pts = np.concatenate([centers + rng.normal(0, 1.5, (3, 3)), rng.uniform(0, L, (60, 3))])
    V = fe.gaussian_potential(pts, L, centers, depth, width)
    ref = _poisson_potential(pts, L, centers, depth, width)
    np.testing.assert_allclose(V, ref, rtol=0, atol=1e-12 * max(depth))
    assert np.abs(V).max() > 0.1      # the sample reaches the wells
