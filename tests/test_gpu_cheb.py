"""GPU parity: Algorithm 2 (paw_cheb_filter) against the oracle's step-by-step
restatement with the same approximate inverse.

The inputs are S-orthonormal Ritz vectors of a random block (iteration 0 of
the R-ChFSI driver), the bounds come from the oracle's dense spectrum.  FP64
agrees to rounding.  FP32: the bracket is rounded to FP32 every step, so
errors relative to the output scale are ~m * 6e-8 * growth of the unwanted
components; 1e-4 bounds them.  TF32 operands: 2e-2 (the filtered block is
still far from converged here, so the residual terms are large).
"""
import numpy as np
import pytest

from oracle import cheb, rr
from tests.gpu_util import gpu_fe, oracle_ops, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4, "tf32": 2e-2}


def _inputs(name, ncols, seed=5):
    op = oracle_ops(name)
    X = np.random.default_rng(seed).standard_normal((op.mesh.ndof, ncols))
    Psi, lam = rr.rayleigh_ritz(op, X)
    tmin, up = rr.lanczos_bounds(lambda x: op.apply_Sinv_exact(op.apply_H(x)), op.apply_S, op.mesh.ndof)
    return op, Psi, lam, (min(lam[0], tmin) - 0.1, lam[-1], up)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32"])
@pytest.mark.parametrize("m", [1, 2, 20])
def test_filter_tiny(prec, m):
    op, Psi, lam, bounds = _inputs("tiny", 16)
    fe = gpu_fe("tiny", block=16)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, m, *bounds)
    out = fe.cheb_filter(to_dev(Psi), lam, m, bounds, prec=prec).cpu().numpy()
    assert rel_err(out, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_filter_blocks_and_ragged_tail(prec):
    """40 columns in blocks of 16 (16 + 16 + 8), degree-6 cells."""
    op, Psi, lam, bounds = _inputs("p6", 40)
    fe = gpu_fe("p6", block=16)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, 8, *bounds)
    out = fe.cheb_filter(to_dev(Psi), lam, 8, bounds, prec=prec).cpu().numpy()
    assert rel_err(out, ref) < TOL[prec]


def test_filter_fixed_point():
    """Exact eigenpairs in: the residual is zero and the output is Psi C_m(Lambda~)."""
    op = oracle_ops("tiny")
    lam, V = rr.dense_eigs(op, 8)
    fe = gpu_fe("tiny", block=8)
    bounds = (lam[0] - 0.05, lam[-1], 95.0)
    out = fe.cheb_filter(to_dev(V), lam, 12, bounds, prec="fp32").cpu().numpy()
    ref = V * cheb.scaled_scalar(12, lam, *bounds)[None, :]
    assert rel_err(out, ref) < 1e-6


def test_filter_rejects_bad_bounds():
    import paper_2604_26037_gb300 as P
    op, Psi, lam, bounds = _inputs("tiny", 4)
    fe = gpu_fe("tiny")
    with pytest.raises(P.PawError) as ei:
        fe.cheb_filter(to_dev(Psi), lam, 5, (1.0, 0.5, 3.0))
    assert ei.value.status == "PAW_ERR_INVALID_ARG"


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_overlapped_blocks_match_serial_schedule(prec):
    """Three blocks (32 + 32 + 16 columns): step 2 of each next block overlaps the loop of the
    current one on two internal streams (the default), or the blocks run one after another.
    Both schedules do the same arithmetic on each column, apart from the order of FP32
    additions, and both match the oracle."""
    op, Psi, lam, bounds = _inputs("p6", 80)
    fe_o = gpu_fe("p6", block=32)
    fe_s = gpu_fe("p6", block=32, overlap=False)
    X = to_dev(Psi)
    out_o = fe_o.cheb_filter(X, lam, 8, bounds, prec=prec)
    out_s = fe_s.cheb_filter(X, lam, 8, bounds, prec=prec)
    fe_o.sync_status()
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, 8, *bounds)
    o, s_ = out_o.cpu().numpy(), out_s.cpu().numpy()
    assert rel_err(o, ref) < TOL[prec] and rel_err(s_, ref) < TOL[prec]
    assert rel_err(o, s_) < (1e-5 if prec == "fp32" else 4e-3)
