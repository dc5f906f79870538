"""Finite-element discretisation for the oracle (FP64, numpy).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Follows Sec. 2.2 (Eq. FEbasisexp: C0 Lagrange basis on GLL nodes) and
Sec. 4.1 (Eq. Quadrature Integration, Eqs. FEM Ham entries, FEM S_loc
entries, FEM Cmatrix) at the Gamma point (k = 0), for a periodic cube of side
L divided into n^3 equal cubic cells of degree p.

Readings taken where the paper leaves a choice open:
* kinetic and mass cell matrices use (p+1)^3 Gauss points (Sec. 4.1 states
  n_q1 = (p+1)^3); the potential and projector integrals use (p+2)^3 Gauss
  points (n_q2, n_q3 are not given numerically).
* M_D is the mass matrix integrated with the GLL rule on the nodes
  (Sec. 3.1, first approximation under Eq. Delta Sinv).
* local node index I = a + n_p (b + n_p c) (x fastest); global DoF of lattice
  point (i, j, k) is i + N1 (j + N1 k) with N1 = n p and periodic wrap.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


# ----------------------------------------------------------------------------
# 1D rules and basis
# ----------------------------------------------------------------------------

def gll_rule(p: int):
    """Gauss-Lobatto-Legendre nodes and weights on [-1, 1] (p+1 points).

    Interior nodes are the roots of P_p'; weights are 2 / (p (p+1) P_p(x)^2).
    Pinned by test_oracle_fe::test_gll_* (exactness up to degree 2p-1,
    textbook values for p = 2, 3).
    """
    Pp = npleg.Legendre.basis(p)
    inner = np.sort(np.real(Pp.deriv().roots()))
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (p * (p + 1) * Pp(x) ** 2)
    return x, w


def gauss_rule(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    x, w = npleg.leggauss(n)
    return x, w


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """Values and derivatives of the Lagrange polynomials on ``nodes`` at x.

    Returns (phi, dphi) with shape (len(x), len(nodes)).
    Pinned by test_oracle_fe::test_lagrange_* (Kronecker property,
    partition of unity, exact derivative of interpolated polynomials).
    """
    nodes = np.asarray(nodes, float)
    x = np.asarray(x, float)
    n = len(nodes)
    phi = np.ones((len(x), n))
    dphi = np.zeros((len(x), n))
    for a in range(n):
        for b in range(n):
            if b != a:
                phi[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        for c in range(n):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b != a and b != c:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            dphi[:, a] += term
    return phi, dphi


# ----------------------------------------------------------------------------
# Mesh
# ----------------------------------------------------------------------------

class Mesh:
    """Periodic cube [0, L)^3 with n^3 cells of Lagrange degree p."""

    def __init__(self, L: float, n: int, p: int):
        self.L, self.n, self.p = float(L), int(n), int(p)
        self.h = self.L / self.n
        self.np1 = p + 1                     # nodes per cell edge
        self.nc = self.np1 ** 3              # nodes per cell
        self.N1 = n * p                      # DoFs per direction
        self.ndof = self.N1 ** 3
        self.ncells = n ** 3
        self.detJ = (self.h / 2.0) ** 3
        self.xi, self.w_gll = gll_rule(p)
        # cell -> global DoF map, shape (ncells, nc)
        a = np.arange(self.np1)
        A, B, C = np.meshgrid(a, a, a, indexing="ij")
        la = A.transpose(2, 1, 0).reshape(-1)   # local index I = a + np1 (b + np1 c)
        lb = B.transpose(2, 1, 0).reshape(-1)
        lc = C.transpose(2, 1, 0).reshape(-1)
        self.local_abc = np.stack([la, lb, lc], 1)
        cells = np.arange(self.ncells)
        cx = cells % n
        cy = (cells // n) % n
        cz = cells // (n * n)
        self.cell_xyz = np.stack([cx, cy, cz], 1)
        gi = (cx[:, None] * p + la[None, :]) % self.N1
        gj = (cy[:, None] * p + lb[None, :]) % self.N1
        gk = (cz[:, None] * p + lc[None, :]) % self.N1
        self.cell_dofs = gi + self.N1 * (gj + self.N1 * gk)

    def node_coords(self) -> np.ndarray:
        """Physical coordinates of every global DoF (ndof, 3)."""
        x1 = np.empty(self.N1)
        for c in range(self.n):
            for a in range(self.p):
                x1[c * self.p + a] = c * self.h + (self.xi[a] + 1.0) * self.h / 2.0
        i = np.arange(self.ndof)
        return np.stack([x1[i % self.N1], x1[(i // self.N1) % self.N1],
                         x1[i // (self.N1 * self.N1)]], 1)

    def quad_points(self, nq1d: int):
        """Physical Gauss points of every cell: (ncells, nq, 3) and weights (nq,)."""
        g, w = gauss_rule(nq1d)
        qi = np.arange(nq1d ** 3)
        i, j, k = qi % nq1d, (qi // nq1d) % nq1d, qi // (nq1d * nq1d)
        ref = np.stack([g[i], g[j], g[k]], 1)             # (nq, 3)
        W = w[i] * w[j] * w[k]
        org = self.cell_xyz * self.h                      # (ncells, 3)
        pts = org[:, None, :] + (ref[None, :, :] + 1.0) * self.h / 2.0
        return pts, W


def basis3d(mesh: Mesh, nq1d: int):
    """3D shape functions N_I and reference gradients at the Gauss points.

    Returns N (nq, nc) and G (3, nq, nc) where G[d] = dN/dxi_d.
    """
    g, _ = gauss_rule(nq1d)
    phi, dphi = lagrange(mesh.xi, g)                      # (nq1d, np1)
    qi = np.arange(nq1d ** 3)
    i, j, k = qi % nq1d, (qi // nq1d) % nq1d, qi // (nq1d * nq1d)
    a, b, c = mesh.local_abc[:, 0], mesh.local_abc[:, 1], mesh.local_abc[:, 2]
    N = phi[i][:, a] * phi[j][:, b] * phi[k][:, c]
    Gx = dphi[i][:, a] * phi[j][:, b] * phi[k][:, c]
    Gy = phi[i][:, a] * dphi[j][:, b] * phi[k][:, c]
    Gz = phi[i][:, a] * phi[j][:, b] * dphi[k][:, c]
    return N, np.stack([Gx, Gy, Gz])


# ----------------------------------------------------------------------------
# Cell matrices (Eqs. FEM Ham entries, FEM S_loc entries)
# ----------------------------------------------------------------------------

def kinetic_cell(mesh: Mesh) -> np.ndarray:
    """K^e_IJ = 1/2 sum_q w_q (J^-1 grad N_I).(J^-1 grad N_J) detJ, (p+1)^3 Gauss.

    Identical for every cell of the uniform mesh.  Pinned by
    test_oracle_fe::test_empty_box_* (separable 3D spectrum) and
    test_kinetic_nullspace.
    """
    N, G = basis3d(mesh, mesh.p + 1)
    _, w = gauss_rule(mesh.p + 1)
    qi = np.arange((mesh.p + 1) ** 3)
    n1 = mesh.p + 1
    W = w[qi % n1] * w[(qi // n1) % n1] * w[qi // (n1 * n1)]
    s = (2.0 / mesh.h) ** 2 * mesh.detJ
    K = np.zeros((mesh.nc, mesh.nc))
    for d in range(3):
        K += G[d].T @ (W[:, None] * G[d])
    return 0.5 * s * K


def mass_cell(mesh: Mesh) -> np.ndarray:
    """M^e_IJ = sum_q w_q N_I N_J detJ with (p+1)^3 Gauss (exact for degree 2p)."""
    N, _ = basis3d(mesh, mesh.p + 1)
    n1 = mesh.p + 1
    _, w = gauss_rule(n1)
    qi = np.arange(n1 ** 3)
    W = w[qi % n1] * w[(qi // n1) % n1] * w[qi // (n1 * n1)]
    return mesh.detJ * (N.T @ (W[:, None] * N))


def lumped_mass(mesh: Mesh) -> np.ndarray:
    """M_D: the mass matrix evaluated with the GLL rule on the nodes (diagonal).

    Assembled cell by cell: every cell adds w_a w_b w_c detJ to the DoF of its
    local node (a, b, c).  Pinned by test_oracle_fe::test_lumped_mass_total.
    """
    w = mesh.w_gll
    a, b, c = mesh.local_abc.T
    cellw = w[a] * w[b] * w[c] * mesh.detJ
    md = np.zeros(mesh.ndof)
    for e in range(mesh.ncells):
        md[mesh.cell_dofs[e]] += cellw
    return md


def gaussian_potential(pts: np.ndarray, L: float, centers, depth, width,
                       image_cut: float = 8.0) -> np.ndarray:
    """V(x) = -sum_atoms sum_images A exp(-|x - R - L n|^2 / (2 w^2)).

    Images within image_cut * w of x contribute (synthetic local potential;
    w is the standard deviation of the Gaussian).  Pinned by
    test_oracle_fe::test_gaussian_potential_values (values at the centre, at
    w and at the cut, wrap-around) and ::test_gaussian_potential_*_poisson
    (both branches against the Poisson-summed periodic Gaussian).
    """
    pts = np.asarray(pts)
    V = np.zeros(pts.shape[:-1])
    for R, A, w in zip(np.asarray(centers), np.asarray(depth), np.asarray(width)):
        rc = image_cut * w
        if rc < L / 2:
            # at most one image lies within rc: the minimum image
            d = pts - R
            d -= L * np.round(d / L)
            r2 = np.sum(d * d, -1)
            V -= np.where(r2 < rc * rc, A * np.exp(-r2 / (2 * w * w)), 0.0)
            continue
        nim = int(math.ceil(rc / L))
        for ix in range(-nim, nim + 1):
            for iy in range(-nim, nim + 1):
                for iz in range(-nim, nim + 1):
                    d = pts - (R + L * np.array([ix, iy, iz]))
                    r2 = np.sum(d * d, -1)
                    V -= np.where(r2 < rc * rc, A * np.exp(-r2 / (2 * w * w)), 0.0)
    return V


def potential_at_quad(mesh: Mesh, sysd: dict) -> np.ndarray:
    """V at the (p+2)^3 Gauss points of every cell, shape (ncells, nq)."""
    pts, _ = mesh.quad_points(mesh.p + 2)
    return gaussian_potential(pts, mesh.L, sysd["vloc_centers"],
                              sysd["vloc_depth"], sysd["vloc_width"])


def vquad_weights(mesh: Mesh) -> np.ndarray:
    """w_q detJ for the (p+2)^3 potential rule."""
    _, W = mesh.quad_points(mesh.p + 2)
    return W * mesh.detJ


def potential_cell(mesh: Mesh, Vq_cell: np.ndarray) -> np.ndarray:
    """V^e_IJ = sum_q w_q V(x_q) N_I N_J detJ for one cell, (p+2)^3 Gauss.

    Pinned by test_oracle_fe::test_constant_potential_shift and
    test_linear_potential_exact.
    """
    N, _ = basis3d(mesh, mesh.p + 2)
    W = vquad_weights(mesh)
    return N.T @ ((W * Vq_cell)[:, None] * N)


# ----------------------------------------------------------------------------
# Projectors (Eqs. FEM Cmatrix, FE nonlocal contribution)
# ----------------------------------------------------------------------------

_SQ = math.sqrt


def solid_harmonics(l: int, d: np.ndarray) -> np.ndarray:
    """r^l Y_lm(r_hat) for m = -l..l (real harmonics, no Condon-Shortley sign).

    d has shape (..., 3); returns (..., 2l+1).  Pinned by
    test_oracle_fe::test_projector_norm (orthonormality on a fine grid).
    """
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    if l == 0:
        return np.full(d.shape[:-1] + (1,), 0.5 / _SQ(math.pi))
    if l == 1:
        c = _SQ(3.0 / (4.0 * math.pi))
        return np.stack([c * y, c * z, c * x], -1)
    if l == 2:
        c1 = 0.5 * _SQ(15.0 / math.pi)
        c0 = 0.25 * _SQ(5.0 / math.pi)
        c2 = 0.25 * _SQ(15.0 / math.pi)
        return np.stack([c1 * x * y, c1 * y * z, c0 * (2 * z * z - x * x - y * y),
                         c1 * x * z, c2 * (x * x - y * y)], -1)
    raise ValueError("l > 2 not supported")


def radial_norm(l: int, w: float) -> float:
    """N_l with int |N_l r^l exp(-r^2/(2w^2)) Y_lm|^2 d^3r = 1."""
    return math.sqrt(2.0 / (math.gamma(l + 1.5) * w ** (2 * l + 3)))


def cutoff_radius(w: float) -> float:
    """Truncation radius w sqrt(2 ln 1e8): the Gaussian factor is 1e-8 there."""
    return w * math.sqrt(2.0 * math.log(1e8))


def projector_values(shells, d: np.ndarray) -> np.ndarray:
    """All projectors of one atom at displacements d (..., 3) -> (..., npj)."""
    out = []
    r2 = np.sum(d * d, -1)
    for l, w in shells:
        rc = cutoff_radius(w)
        g = np.where(r2 < rc * rc, radial_norm(l, w) * np.exp(-r2 / (2 * w * w)), 0.0)
        out.append(solid_harmonics(l, d) * g[..., None])
    return np.concatenate(out, -1)


def min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def projector_overlap_analytic(shells) -> np.ndarray:
    """<p_alpha | p_beta> for projectors on one centre (untruncated), Sec. 3.1."""
    ls, ws = [], []
    for l, w in shells:
        for _m in range(2 * l + 1):
            ls.append(l)
            ws.append(w)
    ms = []
    for l, _ in shells:
        ms.extend(range(-l, l + 1))
    n = len(ls)
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if ls[i] == ls[j] and ms[i] == ms[j]:
                l = ls[i]
                w1, w2 = ws[i], ws[j]
                weff2 = 2 * w1 * w1 * w2 * w2 / (w1 * w1 + w2 * w2)
                G[i, j] = (radial_norm(l, w1) * radial_norm(l, w2) * 0.5
                           * math.gamma(l + 1.5) * weff2 ** (l + 1.5))
    return G


def projector_matrix(mesh: Mesh, sysd: dict, atom: int):
    """Assembled P^a (= C^a of Eq. FE nonlocal contribution) for one atom.

    C^a_{J alpha} = sum_e sum_q w_q N_J(x_q) p_alpha(x_q - R_a) detJ with the
    (p+2)^3 Gauss rule and minimum-image displacements.  Returns
    (dofs, values) with values of shape (len(dofs), npj), dofs sorted.
    Pinned by test_oracle_fe::test_projector_integral.
    """
    shells = sysd["shells"]
    R = np.asarray(sysd["positions"][atom], float)
    rmax = max(cutoff_radius(w) for _, w in shells)
    N, _ = basis3d(mesh, mesh.p + 2)
    pts, W = mesh.quad_points(mesh.p + 2)
    # cells whose centre is within rmax + half diagonal of the atom
    centres = (mesh.cell_xyz + 0.5) * mesh.h
    dc = min_image(centres - R, mesh.L)
    near = np.nonzero(np.linalg.norm(dc, axis=1) < rmax + mesh.h * math.sqrt(3) / 2 + 1e-12)[0]
    npj = sysd["nproj"]
    d = min_image(pts[near] - R, mesh.L)                   # (nnear, nq, 3)
    pv = projector_values(shells, d)                       # (nnear, nq, npj)
    Ce = np.matmul(N.T, (W * mesh.detJ)[None, :, None] * pv)   # C^{e,a}: (nnear, nc, npj)
    alldofs = mesh.cell_dofs[near].reshape(-1)
    dofs, inv = np.unique(alldofs, return_inverse=True)
    vals = np.zeros((len(dofs), npj))
    np.add.at(vals, inv, Ce.reshape(-1, npj))
    return dofs, vals
