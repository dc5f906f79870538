"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import functools

import numpy as np

import inputs
from tests.oracle_systems import mini_system, sym_random


@functools.lru_cache(maxsize=None)
def system(name):
    if name == "tiny":
        return inputs.make_system("tiny")
    if name == "p6":
        # degree-6 cells (343 nodes, like the mid workload) on a small box
        rng = np.random.default_rng(21)
        return mini_system(L=15.0, n=3, p=6, positions=[[2.2, 3.1, 4.4], [8.1, 7.7, 6.2], [5.0, 10.5, 1.2]],
                           shells=[(0, 0.6), (0, 1.2), (1, 0.75), (1, 1.05), (2, 0.9)],
                           D=sym_random(rng, 3, 13, 0.1), dS=sym_random(rng, 3, 13, 0.02),
                           vdepth=2.0, vwidth=1.0)
    if name == "p5":
        rng = np.random.default_rng(22)
        return mini_system(L=10.0, n=3, p=5, positions=[[2.2, 3.1, 4.4], [7.1, 6.7, 6.2]],
                           shells=[(0, 0.7), (1, 0.7), (2, 0.7)],
                           D=sym_random(rng, 2, 9, 0.1), dS=sym_random(rng, 2, 9, 0.02),
                           vdepth=2.0, vwidth=1.0)
    if name == "w18":
        # 18 projectors per atom (two s, two p and two d shells): the projector arrays are
        # padded to 32 instead of 16; the two supports overlap, so the atom-pair Gram blocks
        # between different atoms are non-zero
        rng = np.random.default_rng(23)
        return mini_system(L=10.0, n=3, p=4, positions=[[2.5, 3.0, 4.0], [6.5, 6.0, 5.5]],
                           shells=[(0, 0.6), (0, 0.8), (1, 0.6), (1, 0.8), (2, 0.7), (2, 0.5)],
                           D=sym_random(rng, 2, 18, 0.1), dS=sym_random(rng, 2, 18, 0.02),
                           vdepth=2.0, vwidth=1.0)
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def oracle_ops(name):
    from oracle import ops as O
    return O.PawOperators(system(name))


def gpu_fe(name, **kw):
    import paper_2604_26037_gb300 as P
    return P.PawFE.from_system(system(name), **kw)


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def rel_err(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# measured errors of the parity tests, printed in the terminal summary (tests/conftest.py)
MEASURED = []


def report(test, quantity, value, bound=None):
    MEASURED.append((test, quantity, float(value), None if bound is None else float(bound)))


def gap_index(lam, k0, gap_min=1e-4):
    """State count nearest to k0 with lam[k] - lam[k-1] > gap_min (Ha): compared sets of the
    lowest states never split a (near-)degenerate level (gap-aware choice of k)."""
    n = len(lam)
    for d in range(n):
        for k in (k0 - d, k0 + d):
            if 1 <= k < n and lam[k] - lam[k - 1] > gap_min:
                return k
    return n
