"""GPU parity with 18 projectors per atom (two s, two p and two d shells), so that every
per-atom array is padded to 32 projectors instead of 16: the operator applications and
Algorithm 2 against the oracle, including the fused coupling of the loop (W_S and W_H from
the projections in one launch, with off-diagonal atom-pair blocks since the two supports
overlap) and the overlapped block schedule.  Tolerances as in test_gpu_ops / test_gpu_cheb.
"""
import numpy as np
import pytest

from oracle import cheb, rr
from tests.gpu_util import gpu_fe, oracle_ops, rel_err, system, to_dev

pytestmark = pytest.mark.gpu

TOL_OP = {"fp64": 1e-11, "fp32": 2e-5, "tf32": 4e-3}
TOL_FILTER = {"fp64": 1e-10, "fp32": 1e-4, "tf32": 2e-2}


def _x(op, ncols, seed):
    return np.random.default_rng(seed).standard_normal((op.mesh.ndof, ncols))


def test_projector_count():
    assert system("w18")["nproj"] == 18
    assert oracle_ops("w18").mesh.ndof == 12 ** 3


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32"])
@pytest.mark.parametrize("ncols", [37, 132])
def test_apply_H(prec, ncols):
    import torch
    op, fe = oracle_ops("w18"), gpu_fe("w18")
    X = _x(op, ncols, 1)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Y = fe.apply_H(to_dev(X, dt), prec=prec)
    assert rel_err(Y.double().cpu().numpy(), op.apply_H(X)) < TOL_OP[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32"])
def test_apply_S_and_Sinv(prec):
    import torch
    op, fe = oracle_ops("w18"), gpu_fe("w18")
    X = _x(op, 132, 2)
    dt = torch.float64 if prec == "fp64" else torch.float32
    S = fe.apply_S(to_dev(X, dt), prec=prec)
    assert rel_err(S.double().cpu().numpy(), op.apply_S(X)) < TOL_OP[prec]
    Si = fe.apply_Sinv_approx(to_dev(X, dt), prec=prec)
    assert rel_err(Si.double().cpu().numpy(), op.apply_Sinv_approx(X)) < TOL_OP[prec]


def _inputs(ncols, seed=5):
    op = oracle_ops("w18")
    X = np.random.default_rng(seed).standard_normal((op.mesh.ndof, ncols))
    Psi, lam = rr.rayleigh_ritz(op, X)
    tmin, up = rr.lanczos_bounds(lambda x: op.apply_Sinv_exact(op.apply_H(x)), op.apply_S, op.mesh.ndof)
    return op, Psi, lam, (min(lam[0], tmin) - 0.1, lam[-1], up)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32"])
def test_filter(prec):
    """40 columns in blocks of 16 (16 + 16 + 8), degree 8."""
    op, Psi, lam, bounds = _inputs(40)
    fe = gpu_fe("w18", block=16)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, 8, *bounds)
    out = fe.cheb_filter(to_dev(Psi), lam, 8, bounds, prec=prec)
    fe.sync_status()
    assert rel_err(out.cpu().numpy(), ref) < TOL_FILTER[prec]


def test_filter_overlapped_schedule():
    """Three blocks of 32 + 32 + 16 columns in TF32: overlapped and serial schedules agree."""
    op, Psi, lam, bounds = _inputs(80, seed=6)
    X = to_dev(Psi)
    out_o = gpu_fe("w18", block=32).cheb_filter(X, lam, 8, bounds, prec="tf32")
    out_s = gpu_fe("w18", block=32, overlap=False).cheb_filter(X, lam, 8, bounds, prec="tf32")
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, 8, *bounds)
    o, s_ = out_o.cpu().numpy(), out_s.cpu().numpy()
    assert rel_err(o, ref) < TOL_FILTER["tf32"] and rel_err(s_, ref) < TOL_FILTER["tf32"]
    assert rel_err(o, s_) < 4e-3


@pytest.mark.parametrize("name", ["p6", "w18"])
def test_filter_after_set_dij(name):
    """paw_set_dij after creation: the fused FP32 coupling of the loop (which carries D_H) is
    rebuilt, so the TF32 filter matches the oracle built with the new D_ij."""
    from oracle import ops as O
    from tests.oracle_systems import sym_random
    sysd = dict(system(name))
    D2 = sym_random(np.random.default_rng(31), sysd["natoms"], sysd["nproj"], 0.2)
    sysd["D"] = D2
    op = O.PawOperators(sysd)
    X = np.random.default_rng(7).standard_normal((op.mesh.ndof, 24))
    Psi, lam = rr.rayleigh_ritz(op, X)
    tmin, up = rr.lanczos_bounds(lambda x: op.apply_Sinv_exact(op.apply_H(x)), op.apply_S, op.mesh.ndof)
    bounds = (min(lam[0], tmin) - 0.1, lam[-1], up)
    fe = gpu_fe(name, block=16)
    fe.set_dij(D2)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, 8, *bounds)
    out = fe.cheb_filter(to_dev(Psi), lam, 8, bounds, prec="tf32")
    fe.sync_status()
    assert rel_err(out.cpu().numpy(), ref) < TOL_FILTER["tf32"]
    fe.close()
