"""GPU parity at the full size of the mid workload, in the launch configuration bench.py times.

mid: 884,736 DoFs (16^3 cells of degree 6), 64 atoms x 13 projectors, 512 vectors filtered in
blocks of 256 (the tensor-core kernels' 128-vector tiles), Chebyshev degree 30.  The library
works on all 512 columns; the oracle regenerates two of them on its own (inputs.start_columns
gives every column an independent stream: column 5 of the first block, column 300 of the second)
and computes their outputs on the whole mesh, every row compared.

Tolerances (relative to the largest output entry): operators as in test_gpu_ops / test_gpu_pair32;
the FP64 filter 1e-10 as in test_gpu_cheb; the TF32 filter 5e-2 (random, not Rayleigh-Ritz
rotated start: the residual terms the bracket carries in TF32 are of the size of the vectors,
and degree 30 compounds their rounding; the tiny workload at degree 20 from Ritz vectors keeps
2e-2).
"""
import functools

import numpy as np
import pytest

import inputs
from tests.gpu_util import rel_err, report, to_dev

pytestmark = pytest.mark.gpu

NAME = "mid"
COLS = (5, 300)


@functools.lru_cache(maxsize=None)
def _oracle():
    from oracle import ops as O
    return O.PawOperators(inputs.make_system(NAME))


@functools.lru_cache(maxsize=None)
def _fe(pair32=False):
    import paper_2604_26037_gb300 as P
    cfg = inputs.CONFIGS[NAME]
    return P.PawFE.from_system(inputs.make_system(NAME), block=cfg["block"], y0_pair32=pair32)


@functools.lru_cache(maxsize=None)
def _X():
    cfg = inputs.CONFIGS[NAME]
    return to_dev(inputs.start_columns(NAME, range(cfg["nvec"])))


def _lam():
    return np.linspace(-0.3, 0.2, inputs.CONFIGS[NAME]["nvec"])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("f32x2", 5e-12), ("tf32", 4e-3)])
def test_operators_full_size(prec, tol):
    import torch
    fe, op = _fe(), _oracle()
    X = _X()
    Xs = inputs.start_columns(NAME, COLS)
    Xin = X if prec in ("fp64", "f32x2") else X.float()
    H = fe.apply_H(Xin, prec=prec)[:, list(COLS)].double().cpu().numpy()
    S = fe.apply_S(Xin, prec=prec)[:, list(COLS)].double().cpu().numpy()
    errs = {"H": rel_err(H, op.apply_H(Xs)), "S": rel_err(S, op.apply_S(Xs))}
    if prec != "f32x2":
        Si = fe.apply_Sinv_approx(Xin, prec=prec)[:, list(COLS)].double().cpu().numpy()
        errs["Sinv"] = rel_err(Si, op.apply_Sinv_approx(Xs))
    for k, v in errs.items():
        report(f"mid operators {prec}", f"{k} relative error", v, tol)
    assert max(errs.values()) < tol
    del H, S
    torch.cuda.empty_cache()


@functools.lru_cache(maxsize=None)
def _oracle_filter(bounds):
    from oracle import cheb
    op = _oracle()
    m = inputs.CONFIGS[NAME]["degree"]
    lam = _lam()[list(COLS)]
    return cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, inputs.start_columns(NAME, COLS),
                              lam, m, *bounds)


@functools.lru_cache(maxsize=None)
def _bounds():
    tmin, bU = _fe().lanczos_bounds(20, 7)
    return (min(-0.3, tmin), 0.2, float(bU))


@pytest.mark.parametrize("prec,pair32,tol", [("fp64", False, 1e-10), ("tf32", False, 5e-2),
                                             ("tf32", True, 5e-2)])
def test_filter_full_size(prec, pair32, tol):
    """Algorithm 2 on all 512 columns (two 256-column blocks) against the oracle's two columns."""
    import torch
    fe = _fe(pair32)
    bounds = _bounds()
    m = inputs.CONFIGS[NAME]["degree"]
    out = fe.cheb_filter(_X(), _lam(), m, bounds, prec=prec)
    got = out[:, list(COLS)].cpu().numpy()
    del out
    torch.cuda.empty_cache()
    err = rel_err(got, _oracle_filter(bounds))
    report(f"mid filter {prec}{' pair32 step 2' if pair32 else ''}", "relative error", err, tol)
    assert err < tol


def test_filter_calls_are_stream_ordered():
    """Two TF32 filter calls on one stream, no host wait between them: each returns once its
    work is enqueued (the stream is still busy when the second returns), and both outputs
    match the oracle's columns."""
    import torch
    fe = _fe()
    bounds = _bounds()
    m = inputs.CONFIGS[NAME]["degree"]
    X = _X()
    torch.cuda.synchronize()
    out1 = fe.cheb_filter(X, _lam(), m, bounds, prec="tf32")
    out2 = fe.cheb_filter(X, _lam(), m, bounds, prec="tf32")
    busy = not torch.cuda.current_stream().query()
    fe.sync_status()
    ref = _oracle_filter(bounds)
    e1 = rel_err(out1[:, list(COLS)].cpu().numpy(), ref)
    e2 = rel_err(out2[:, list(COLS)].cpu().numpy(), ref)
    del out1, out2
    torch.cuda.empty_cache()
    report("mid filter tf32, two calls without a host wait", "relative error (first, second)", max(e1, e2), 5e-2)
    assert busy, "the second call returned after the GPU had finished both"
    assert e1 < 5e-2 and e2 < 5e-2
