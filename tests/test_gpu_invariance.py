"""GPU: the library's operators and filter under the symmetries of the problem.

Numbering the atoms differently changes the owner-cell pair lists, the order of
the per-atom sums and every tensor-core image of the projectors, but not H, S
or Shat^-1; moving every atom by whole cells of the periodic box moves every
result by the same number of nodes (DoF i + N1 (j + N1 k)).  FP64 forms agree
to rounding (1e-12 of the largest entry; the filter, m = 4, 1e-10); the TF32
forms sum their FP32 tiles in another order, 1e-4.
"""
import numpy as np
import pytest

import inputs
from tests.gpu_util import rel_err, system, to_dev
from tests.oracle_systems import reorder_atoms, shift_nodes, translate_cells

pytestmark = pytest.mark.gpu


def _systems():
    return {"p6": system("p6"), "small6": inputs.make_system("small6")}


def _fe(sysd):
    import paper_2604_26037_gb300 as P
    return P.PawFE.from_system(sysd, block=64)


@pytest.fixture(scope="module", params=["p6", "small6"])
def case(request):
    sysd = _systems()[request.param]
    base = _fe(sysd)
    na = int(sysd["natoms"])
    order = list(range(na))[::-1] if na > 2 else [1, 0]
    perm = _fe(reorder_atoms(sysd, order))
    cells = (1, 2, 0) if sysd["ncell"] > 2 else (1, 2, 1)
    moved = _fe(translate_cells(sysd, cells))
    yield request.param, sysd, base, perm, moved, cells
    for h in (base, perm, moved):
        h.close()


@pytest.mark.parametrize("op", ["apply_H", "apply_S", "apply_Sinv_approx"])
def test_atom_order_and_translation_fp64(case, op):
    import torch
    name, sysd, base, perm, moved, cells = case
    X = np.random.default_rng(5).standard_normal((sysd["ndof"], 37))
    ref = getattr(base, op)(to_dev(X, torch.float64), prec="fp64").cpu().numpy()
    out_p = getattr(perm, op)(to_dev(X, torch.float64), prec="fp64").cpu().numpy()
    assert rel_err(out_p, ref) < 1e-12, (name, op, "atom order")
    PX = shift_nodes(X, sysd, cells)
    out_t = getattr(moved, op)(to_dev(PX, torch.float64), prec="fp64").cpu().numpy()
    assert rel_err(out_t, shift_nodes(ref, sysd, cells)) < 1e-12, (name, op, "translation")


def test_atom_order_and_translation_tf32(case):
    """132 columns: the tensor-core cell and projector kernels."""
    import torch
    name, sysd, base, perm, moved, cells = case
    X = np.random.default_rng(6).standard_normal((sysd["ndof"], 132))
    ref = base.apply_H(to_dev(X, torch.float32), prec="tf32").double().cpu().numpy()
    out_p = perm.apply_H(to_dev(X, torch.float32), prec="tf32").double().cpu().numpy()
    assert rel_err(out_p, ref) < 1e-4, (name, "atom order")
    PX = shift_nodes(X, sysd, cells)
    out_t = moved.apply_H(to_dev(PX, torch.float32), prec="tf32").double().cpu().numpy()
    assert rel_err(out_t, shift_nodes(ref, sysd, cells)) < 1e-4, (name, "translation")


def test_filter_translation_fp64(case):
    import torch
    name, sysd, base, perm, moved, cells = case
    X = np.random.default_rng(7).standard_normal((sysd["ndof"], 20))
    lam = np.linspace(-0.5, 0.3, 20)
    bounds = (-0.7, 0.35, 150.0)
    ref = base.cheb_filter(to_dev(X, torch.float64), lam, 4, bounds, prec="fp64").cpu().numpy()
    out = moved.cheb_filter(to_dev(shift_nodes(X, sysd, cells), torch.float64), lam, 4, bounds,
                            prec="fp64").cpu().numpy()
    assert rel_err(out, shift_nodes(ref, sysd, cells)) < 1e-10, name
