"""Seeded synthetic inputs for the PAW-FE Chebyshev-filter workloads.

This module only draws random numbers and lays out the workload descriptions
(box, mesh, atoms, projector shells, coupling matrices, start vectors).  It
holds none of the finite-element or eigensolver arithmetic: both the CPU
oracle and the CUDA library receive exactly these arrays and build every
operator themselves.

Workloads (periodic cubes with uniform hexahedral cells):

* ``tiny``    L = 10 bohr, 4^3 cells of degree 4 (16^3 DoFs), 2 atoms with
              4 projectors (l = 0, 1; Gaussian width 0.8 bohr), 16 vectors,
              Chebyshev degree 20, 10 R-ChFSI iterations, 8 wanted states.
* ``mid``     L = 40 bohr, 16^3 cells of degree 6 (96^3 = 884,736 DoFs),
              64 atoms on a jittered 4^3 lattice, 13 projectors each,
              512 vectors in blocks of 256, Chebyshev degree 30.
* ``large``   L = 60 bohr, 24^3 cells of degree 6 (144^3 DoFs), 256 atoms on
              a jittered 8x8x4 lattice, 3000 vectors in blocks of 512,
              Chebyshev degree 40.
* ``grad16``  the ``mid`` atom set at the ``tiny`` resolution (h = 2.5 bohr,
              degree 4): 16^3 cells, 64^3 DoFs, 16 vectors.
* batched     ``batch_systems()``: independent instances of uneven size, cell
              size h = 2.5 bohr (L = 2.5 n, n drawn from a range), degree drawn
              from a set, seeded uniform atom positions, block widths drawn
              from {32, ..., 512}; see its docstring for the caps.

The local potential is a sum of attractive Gaussians
V(r) = -A exp(-r^2 / (2 w^2)) (A = 2 Ha, w = 1 bohr), one per atom.
Projector shells are (l, width) pairs; a shell with angular momentum l
contributes 2l + 1 projectors (m = -l..l).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2604026037

# stream ids inside one workload
_S_POS, _S_D, _S_DS, _S_X, _S_LAMBDA = 0, 1, 2, 3, 4

CONFIGS = {
    "tiny": dict(index=0, L=10.0, ncell=4, p=4, natoms=2,
                 shells=[(0, 0.8), (1, 0.8)], lattice=None, min_sep=3.0,
                 nvec=16, block=16, degree=20, iters=10, nwanted=8),
    "mid": dict(index=1, L=40.0, ncell=16, p=6, natoms=64,
                shells=[(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)],
                lattice=(4, 4, 4), jitter=0.3,
                nvec=512, block=256, degree=30, iters=1, nwanted=512),
    "large": dict(index=2, L=60.0, ncell=24, p=6, natoms=256,
                  shells=[(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)],
                  lattice=(8, 8, 4), jitter=0.3,
                  nvec=3000, block=512, degree=40, iters=1, nwanted=3000),
    # small degree-6 case for profiler captures (same cell size and projector set as mid)
    "small6": dict(index=5, L=20.0, ncell=8, p=6, natoms=8,
                   shells=[(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)],
                   lattice=(2, 2, 2), jitter=0.3,
                   nvec=256, block=256, degree=4, iters=1, nwanted=256),
    # moderate case for profiler captures: arrays of 128 vectors (191 MB) exceed L2,
    # the whole problem holds a few GB on the device
    "prof12": dict(index=6, L=30.0, ncell=12, p=6, natoms=27,
                   shells=[(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)],
                   lattice=(3, 3, 3), jitter=0.3,
                   nvec=128, block=128, degree=4, iters=1, nwanted=128),
    "grad16": dict(index=4, L=40.0, ncell=16, p=4, natoms=64,
                   shells=[(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)],
                   lattice=(4, 4, 4), jitter=0.3,
                   nvec=16, block=16, degree=20, iters=1, nwanted=16),
}

VLOC_DEPTH = 2.0      # Ha
VLOC_WIDTH = 1.0      # bohr (standard deviation of the Gaussian)
D_SIGMA = 0.1         # standard deviation of the Delta_H entries
DS_SIGMA = 0.02       # standard deviation of the Delta_S entries


def _rng(cfg_index: int, stream: int, sub: int = 0, seed: int = BASE_SEED):
    ss = np.random.SeedSequence(entropy=seed, spawn_key=(cfg_index, stream, sub))
    return np.random.Generator(np.random.PCG64(ss))


def nproj_of(shells) -> int:
    return int(sum(2 * l + 1 for l, _ in shells))


def _positions(cfg, rng):
    L = cfg["L"]
    n = cfg["natoms"]
    if cfg.get("lattice") is not None:
        nx, ny, nz = cfg["lattice"]
        sp = np.array([L / nx, L / ny, L / nz])
        grid = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                                    indexing="ij"), -1).reshape(-1, 3)
        pos = (grid + 0.5) * sp
        pos = pos + rng.uniform(-cfg["jitter"], cfg["jitter"], size=pos.shape)
        assert pos.shape[0] == n
        return np.mod(pos, L)
    # uniform positions with a minimum (periodic) separation, by rejection
    pos = []
    while len(pos) < n:
        cand = rng.uniform(0.0, L, size=3)
        ok = True
        for q in pos:
            d = cand - q
            d -= L * np.round(d / L)
            if np.linalg.norm(d) < cfg["min_sep"]:
                ok = False
                break
        if ok:
            pos.append(cand)
    return np.array(pos)


def _sym(rng, n, sigma, count):
    out = np.empty((count, n, n))
    for a in range(count):
        u = rng.normal(0.0, sigma, size=(n, n))
        out[a] = np.triu(u) + np.triu(u, 1).T
    return out


def make_system(name: str, seed: int = BASE_SEED) -> dict:
    """Return the seeded description of one workload (no vectors)."""
    return _build(dict(CONFIGS[name]), name, seed)


def _build(cfg: dict, name: str, seed: int) -> dict:
    idx = cfg["index"]
    pos = _positions(cfg, _rng(idx, _S_POS, seed=seed))
    npj = nproj_of(cfg["shells"])
    D = _sym(_rng(idx, _S_D, seed=seed), npj, D_SIGMA, cfg["natoms"])
    dS = _sym(_rng(idx, _S_DS, seed=seed), npj, DS_SIGMA, cfg["natoms"])
    cfg.update(
        name=name,
        positions=pos,
        nproj=npj,
        D=D,
        dS=dS,
        vloc_centers=pos.copy(),
        vloc_depth=np.full(cfg["natoms"], VLOC_DEPTH),
        vloc_width=np.full(cfg["natoms"], VLOC_WIDTH),
        ndof=(cfg["ncell"] * cfg["p"]) ** 3,
    )
    return cfg


BASE_SHELLS = [(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)]
_TRUNC = float(np.sqrt(2.0 * np.log(1e8)))   # projector cutoff radius / width


def batch_systems(count: int = 32, n_range=(4, 12), degrees=(4, 5, 6), atoms_range=(8, 64),
                  widths=(32, 64, 128, 256, 512), degree: int = 25,
                  seed: int = BASE_SEED) -> list:
    """Seeded independent instances for the batched filter.

    Instance i: n ~ U{n_range}, L = 2.5 n, p ~ U(degrees), the five projector
    shells of the mid workload (13 projectors), B ~ U(widths) vectors, filter
    degree `degree`.  Atoms are placed uniformly with a minimum periodic
    separation of 2.5 bohr; their count is drawn from atoms_range.  Two
    geometric caps keep every instance valid: the shell widths are scaled by
    min(1, 0.45 L / r_c,max) so that every cutoff radius stays below L/2
    (minimum image), and the atom count is at most L^3 / 30 (spheres of the
    minimum separation fill 27% of the box, below the 38% at which random
    sequential placement jams; only the 10 bohr boxes are capped, at 33).
    """
    rng = _rng(99, 0, seed=seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        p = int(rng.choice(np.asarray(degrees)))
        L = 2.5 * n
        rc_max = max(w for _, w in BASE_SHELLS) * _TRUNC
        scale = min(1.0, 0.45 * L / rc_max)
        shells = [(l, w * scale) for l, w in BASE_SHELLS]
        cap = int(min(atoms_range[1], L ** 3 / 30.0))
        natoms = int(rng.integers(atoms_range[0], max(atoms_range[0], cap) + 1))
        B = int(rng.choice(np.asarray(widths)))
        cfg = dict(index=100 + i, L=L, ncell=n, p=p, natoms=natoms, shells=shells, lattice=None,
                   min_sep=2.5, nvec=B, block=B, degree=degree, iters=1, nwanted=B)
        out.append(_build(cfg, f"batch{i}", seed))
    return out


def _atoms_per_cell(pos, L, n, rc):
    """Largest number of atoms whose projectors reach the owned nodes of one cell.

    A cell carries an atom's projector block when its centre lies within
    rc + h sqrt(3)/2 of the atom (periodic); the nodes a cell owns (local
    indices < p) are shared with its neighbours in the -x, -y, -z directions,
    so the count runs over the support cells shifted by 0 or 1 cell per axis.
    """
    h = L / n
    idx = np.arange(n)
    cz, cy, cx = np.meshgrid(idx, idx, idx, indexing="ij")
    centers = np.stack([cx, cy, cz], -1).reshape(-1, 3) * h + h / 2
    count = np.zeros((n, n, n), int)
    reach = rc + h * np.sqrt(3.0) / 2.0
    for x in np.asarray(pos):
        d = centers - x
        d -= L * np.round(d / L)
        sup = (np.sqrt((d ** 2).sum(1)) < reach).reshape(n, n, n)   # [cz][cy][cx]
        own = np.zeros_like(sup)
        for sz in (0, 1):
            for sy in (0, 1):
                for sx in (0, 1):
                    own |= np.roll(sup, (sz, sy, sx), axis=(0, 1, 2))
        count += own
    return int(count.max())


def columns_of(sysd: dict, cols, seed: int = BASE_SEED) -> np.ndarray:
    """start_columns for a system description (also the batched instances)."""
    ndof = sysd["ndof"]
    cols = list(cols)
    out = np.empty((ndof, len(cols)))
    for j, c in enumerate(cols):
        out[:, j] = _rng(sysd["index"], _S_X, int(c), seed=seed).standard_normal(ndof)
    return out


def start_columns(name: str, cols, ndof: int | None = None,
                  seed: int = BASE_SEED) -> np.ndarray:
    """Random N(0,1) start vectors, one independent stream per column.

    Returns an (ndof, len(cols)) float64 array, DoF-major with the vector
    index fastest.  Any subset of columns can be regenerated on its own.
    """
    cfg = CONFIGS[name]
    if ndof is None:
        ndof = (cfg["ncell"] * cfg["p"]) ** 3
    cols = list(cols)
    out = np.empty((ndof, len(cols)))
    for j, c in enumerate(cols):
        out[:, j] = _rng(cfg["index"], _S_X, int(c), seed=seed).standard_normal(ndof)
    return out


def random_lambda(name: str, n: int, lo: float, hi: float,
                  seed: int = BASE_SEED) -> np.ndarray:
    """Sorted uniform eigenvalue guesses in [lo, hi] (for operator tests)."""
    cfg = CONFIGS[name]
    return np.sort(_rng(cfg["index"], _S_LAMBDA, seed=seed).uniform(lo, hi, size=n))
