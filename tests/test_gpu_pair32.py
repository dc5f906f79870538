"""GPU parity of the pair-of-FP32 arithmetic (PAW_F32X2) against the FP64 oracle.

H and S applied with every product and sum in two-FP32 arithmetic (a value is
hi + lo, about 48 significant bits), and Algorithm 2 with its step 2
(Y = H X - S X Lambda) formed that way (options.y0_pair32).

Tolerance of the operators: each output is a chain of six 1D contractions of
<= 10 terms; every pair operation rounds at most about 2^-46 of the magnitudes
it sums, so 5e-12 of the largest output entry bounds the chain with room for
the cancellation inside the 1D stiffness products (FP64 rounds about 30x
finer; FP32 storage would give 1e-6).  The filter with the FP64 bracket keeps
the FP64 tolerance of test_gpu_cheb.
"""
import numpy as np
import pytest

from oracle import cheb, rr
from tests.gpu_util import gpu_fe, oracle_ops, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL_OP = 5e-12


@pytest.fixture(scope="module", params=["tiny", "p6", "p5"])
def pair(request):
    return request.param, oracle_ops(request.param), gpu_fe(request.param)


@pytest.mark.parametrize("ncols", [1, 37, 64])
def test_pair_arithmetic_H_and_S(pair, ncols):
    """ncols 1, a ragged 37 (tail of a 32-vector tile) and 64 on p = 4, 5, 6."""
    name, op, fe = pair
    X = np.random.default_rng(31).standard_normal((op.mesh.ndof, ncols))
    Xd = to_dev(X)
    H = fe.apply_H(Xd, prec="f32x2").cpu().numpy()
    S = fe.apply_S(Xd, prec="f32x2").cpu().numpy()
    assert rel_err(H, op.apply_H(X)) < TOL_OP
    assert rel_err(S, op.apply_S(X)) < TOL_OP
    # the FP64 kernels on the same input: the two forms differ only by rounding
    assert rel_err(H, fe.apply_H(Xd, prec="fp64").cpu().numpy()) < TOL_OP


def test_pair_arithmetic_strided_and_empty(pair):
    """A column block of a wider array (ld > ncols) and ncols = 0."""
    import torch
    name, op, fe = pair
    X = np.random.default_rng(32).standard_normal((op.mesh.ndof, 40))
    big = to_dev(X)
    Yfull = torch.full((op.mesh.ndof, 40), 7.0, dtype=torch.float64, device="cuda")
    fe.apply_H(big[:, 5:17], Y=Yfull[:, 10:22], prec="f32x2")
    out = Yfull.cpu().numpy()
    assert rel_err(out[:, 10:22], op.apply_H(X[:, 5:17])) < TOL_OP
    assert np.all(out[:, :10] == 7.0) and np.all(out[:, 22:] == 7.0)
    fe.apply_H(big[:, :0], Y=Yfull[:, :0], prec="f32x2")


def _filter_inputs(name, ncols, seed=5):
    op = oracle_ops(name)
    X = np.random.default_rng(seed).standard_normal((op.mesh.ndof, ncols))
    Psi, lam = rr.rayleigh_ritz(op, X)
    tmin, up = rr.lanczos_bounds(lambda x: op.apply_Sinv_exact(op.apply_H(x)), op.apply_S, op.mesh.ndof)
    return op, Psi, lam, (min(lam[0], tmin) - 0.1, lam[-1], up)


@pytest.mark.parametrize("name,ncols,block,m", [("tiny", 16, 16, 20), ("p6", 40, 16, 8)])
def test_filter_with_pair_step2(name, ncols, block, m):
    """Algorithm 2 with the FP64 bracket and a pair-arithmetic step 2 against the
    oracle (p6: blocks 16 + 16 + 8); TF32 bracket within its own tolerance."""
    op, Psi, lam, bounds = _filter_inputs(name, ncols)
    fe = gpu_fe(name, block=block, y0_pair32=True)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, Psi, lam, m, *bounds)
    out = fe.cheb_filter(to_dev(Psi), lam, m, bounds, prec="fp64").cpu().numpy()
    assert rel_err(out, ref) < 1e-10
    out = fe.cheb_filter(to_dev(Psi), lam, m, bounds, prec="tf32").cpu().numpy()
    assert rel_err(out, ref) < 2e-2
    fe.close()


def test_pair_rejections():
    import paper_2604_26037_gb300 as P
    from tests.gpu_util import system
    fe = gpu_fe("tiny")
    X = to_dev(np.ones((fe.ndof, 2)))
    with pytest.raises(P.PawError, match="PAW_ERR_UNSUPPORTED"):
        fe.apply_Sinv_approx(X, prec="f32x2")
    with pytest.raises(P.PawError, match="PAW_ERR_UNSUPPORTED"):
        P.PawFE.from_system(system("tiny"), kpoint=(0.1, 0.0, 0.0), y0_pair32=True)
    kfe = P.PawFE.from_system(system("tiny"), kpoint=(0.1, 0.0, 0.0))
    Xc = to_dev(np.ones((kfe.ndof, 2)) + 0j)
    with pytest.raises(P.PawError, match="PAW_ERR_UNSUPPORTED"):
        kfe.apply_H(Xc, prec="f32x2")
    kfe.close()
