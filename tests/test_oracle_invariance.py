"""Pins of the oracle by symmetries of the problem.

H and S are sums over atoms (Eq. FE nonlocal contribution) and over cells
(Eqs. FEM Ham entries, FEM S_loc entries), and the box is periodic: numbering
the atoms differently changes no result, and moving every atom (with its
potential) by whole cells moves every result by the same number of nodes.
A mix-up of atom indices between projectors and D_ij / Delta S_ij, or a wrong
periodic image of a potential or a projector, breaks one of these.
"""
import numpy as np
import pytest

from oracle import ops as O
from tests.oracle_systems import mini_system, reorder_atoms, shift_nodes, sym_random, translate_cells


def _three_atoms(seed=11):
    rng = np.random.default_rng(seed)
    pos = [[1.3, 8.7, 2.2], [6.9, 4.1, 7.6], [4.4, 1.0, 9.3]]   # near faces: images matter
    D = sym_random(rng, 3, 4, 0.1)
    dS = sym_random(rng, 3, 4, 0.02)
    return mini_system(L=10.0, n=4, p=3, positions=pos, shells=[(0, 0.8), (1, 0.8)], D=D, dS=dS,
                       vdepth=2.0, vwidth=1.0)


def _ops(op):
    return {"H": op.apply_H, "S": op.apply_S, "Sinv": op.apply_Sinv_approx, "Sinv_exact": op.apply_Sinv_exact}


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_atom_numbering_changes_nothing():
    sysd = _three_atoms()
    base = _ops(O.PawOperators(sysd))
    X = np.random.default_rng(1).standard_normal((sysd["ndof"], 3))
    for order in ((2, 0, 1), (1, 0, 2)):
        perm = _ops(O.PawOperators(reorder_atoms(sysd, order)))
        for name in base:
            assert _rel(perm[name](X), base[name](X)) < 1e-12, (order, name)


@pytest.mark.parametrize("cells", [(1, 0, 0), (0, 3, 1), (2, 1, 3)])
def test_translation_by_whole_cells(cells):
    sysd = _three_atoms()
    base = _ops(O.PawOperators(sysd))
    moved = _ops(O.PawOperators(translate_cells(sysd, cells)))
    X = np.random.default_rng(2).standard_normal((sysd["ndof"], 2))
    PX = shift_nodes(X, sysd, cells)
    for name in base:
        assert _rel(moved[name](PX), shift_nodes(base[name](X), sysd, cells)) < 1e-11, (cells, name)


def test_translation_pin_detects_a_half_cell_shift():
    """The pin is not vacuous: moving the atoms by half a cell does not commute with a
    shift of the nodes (the potential and projectors sample the basis differently)."""
    sysd = _three_atoms()
    base = O.PawOperators(sysd)
    half = O.PawOperators(translate_cells(sysd, (0.5, 0, 0)))
    X = np.random.default_rng(3).standard_normal((sysd["ndof"], 1))
    cells = (1, 0, 0)   # the nearest whole-node shift of the lattice (p nodes per cell)
    assert _rel(half.apply_H(shift_nodes(X, sysd, cells)), shift_nodes(base.apply_H(X), sysd, cells)) > 1e-3
