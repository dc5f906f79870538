"""GPU parity: operator applications (H, S, approximate S^-1) against the oracle.

Tolerances: FP64 forms agree to rounding (1e-11 relative to the largest output
entry).  FP32 storage with FP32 FMA: each output entry is a sum of <= 8*343
products with unit roundoff 6e-8, so 2e-5 of the largest entry.  TF32 operands
(10-bit mantissa, unit roundoff 4.9e-4 on each operand) give 4e-3.
"""
import numpy as np
import pytest

from tests.gpu_util import gpu_fe, oracle_ops, rel_err, system, to_dev

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 2e-5, "tf32": 4e-3, "bf16": 3e-2}


@pytest.fixture(scope="module", params=["tiny", "p6", "p5"])
def pair(request):
    return request.param, oracle_ops(request.param), gpu_fe(request.param)


def _x(op, ncols, seed):
    return np.random.default_rng(seed).standard_normal((op.mesh.ndof, ncols))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
@pytest.mark.parametrize("ncols", [1, 37, 130, 132, 256])
def test_apply_H(pair, prec, ncols):
    """ncols 132 and 256 take the tensor-core cell and projector kernels
    (column count a multiple of 4); 132 leaves a 4-vector tail tile."""
    import torch
    name, op, fe = pair
    X = _x(op, ncols, 1)
    ref = op.apply_H(X)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Y = fe.apply_H(to_dev(X, dt), prec=prec)
    assert rel_err(Y.double().cpu().numpy(), ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_S_and_Sinv(pair, prec):
    import torch
    name, op, fe = pair
    X = _x(op, 19, 2)
    dt = torch.float64 if prec == "fp64" else torch.float32
    S = fe.apply_S(to_dev(X, dt), prec=prec)
    assert rel_err(S.double().cpu().numpy(), op.apply_S(X)) < TOL[prec]
    Si = fe.apply_Sinv_approx(to_dev(X, dt), prec=prec)
    assert rel_err(Si.double().cpu().numpy(), op.apply_Sinv_approx(X)) < TOL[prec]


def test_strided_block_and_empty(pair):
    """A column block of a wider array (ld > ncols) and ncols = 0."""
    import torch
    name, op, fe = pair
    X = _x(op, 40, 3)
    big = to_dev(X)
    Yfull = torch.full((op.mesh.ndof, 40), 7.0, dtype=torch.float64, device="cuda")
    fe.apply_H(big[:, 5:17], Y=Yfull[:, 10:22])
    ref = op.apply_H(X[:, 5:17])
    out = Yfull.cpu().numpy()
    assert rel_err(out[:, 10:22], ref) < 1e-11
    assert np.all(out[:, :10] == 7.0) and np.all(out[:, 22:] == 7.0)
    fe.apply_H(big[:, :0], Y=Yfull[:, :0])


def test_info(pair):
    name, op, fe = pair
    s = system(name)
    assert fe.ndof == op.mesh.ndof
    assert fe.nodes_per_cell == (s["p"] + 1) ** 3
    assert fe.quad_per_cell == (s["p"] + 2) ** 3
