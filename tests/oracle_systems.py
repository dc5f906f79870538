"""Small hand-built systems for the oracle pin tests (no randomness beyond seeds)."""
import numpy as np


def mini_system(L=10.0, n=2, p=3, positions=(), shells=((0, 0.8), (1, 0.8)),
                D=None, dS=None, vdepth=0.0, vwidth=1.0, vcenters=None):
    positions = np.array(positions, float).reshape(-1, 3)
    na = len(positions)
    npj = sum(2 * l + 1 for l, _ in shells)
    if D is None:
        D = np.zeros((na, npj, npj))
    if dS is None:
        dS = np.zeros((na, npj, npj))
    vc = positions if vcenters is None else np.array(vcenters, float).reshape(-1, 3)
    return dict(L=L, ncell=n, p=p, natoms=na, nproj=npj, shells=list(shells),
                positions=positions, D=np.asarray(D, float), dS=np.asarray(dS, float),
                vloc_centers=vc, vloc_depth=np.full(len(vc), vdepth),
                vloc_width=np.full(len(vc), vwidth), ndof=(n * p) ** 3)


def sym_random(rng, na, npj, sigma):
    out = np.empty((na, npj, npj))
    for a in range(na):
        u = rng.normal(0, sigma, (npj, npj))
        out[a] = 0.5 * (u + u.T)
    return out


def reorder_atoms(sysd, order):
    """The same system with its atoms (and their potentials) numbered in `order`."""
    s = dict(sysd)
    for k in ("positions", "D", "dS", "vloc_centers", "vloc_depth", "vloc_width"):
        s[k] = np.asarray(sysd[k])[list(order)].copy()
    return s


def translate_cells(sysd, cells):
    """Every atom and potential centre moved by `cells` whole cells (periodic box)."""
    s = dict(sysd)
    h = sysd["L"] / sysd["ncell"]
    d = h * np.asarray(cells, float)
    s["positions"] = np.mod(np.asarray(sysd["positions"]) + d, sysd["L"])
    s["vloc_centers"] = np.mod(np.asarray(sysd["vloc_centers"]) + d, sysd["L"])
    return s


def shift_nodes(X, sysd, cells):
    """Nodal vectors moved with the atoms by `cells` whole cells:
    (Pi x)[i, j, k] = x[i - cx p, j - cy p, k - cz p] (DoF i + N1 (j + N1 k), N1 = n p)."""
    N1 = sysd["ncell"] * sysd["p"]
    p = sysd["p"]
    Xr = np.asarray(X).reshape(N1, N1, N1, -1)            # [k][j][i][column]
    Xr = np.roll(Xr, (cells[2] * p, cells[1] * p, cells[0] * p), axis=(0, 1, 2))
    return Xr.reshape(N1 ** 3, -1)
