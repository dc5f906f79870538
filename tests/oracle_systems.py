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
