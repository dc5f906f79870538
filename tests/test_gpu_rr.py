"""GPU parity: Rayleigh-Ritz, residual norms, Lanczos bounds and the full
R-ChFSI iteration (Algorithm 1 with Algorithm 2) on the tiny workload."""
import numpy as np
import pytest

import inputs
from oracle import rr
from tests.gpu_util import gpu_fe, oracle_ops, rel_err, to_dev

pytestmark = pytest.mark.gpu


def test_rayleigh_ritz_and_residuals():
    op = oracle_ops("tiny")
    X = np.random.default_rng(8).standard_normal((op.mesh.ndof, 12))
    Psi_ref, lam_ref = rr.rayleigh_ritz(op, X)
    fe = gpu_fe("tiny")
    Xd = to_dev(X)
    lam = fe.rayleigh_ritz(Xd)
    assert np.abs(lam - lam_ref).max() < 1e-10 * max(1, np.abs(lam_ref).max())
    # Ritz vectors agree up to sign (no degenerate Ritz values for a random block)
    Psi = Xd.cpu().numpy()
    sgn = np.sign(np.sum(Psi * Psi_ref, 0))
    assert rel_err(Psi * sgn, Psi_ref) < 1e-8
    r = fe.residuals(Xd, lam)
    r_ref = rr.residual_norms(op, Psi_ref, lam_ref)
    assert np.abs(r - r_ref).max() < 1e-9 * r_ref.max()


def test_rayleigh_ritz_mixed_rotation():
    """rr_mixed: the projected problem is the same FP64 one (same Ritz values); the
    rotation uses FP64 for diag(Q) and an FP32 GEMM for the rest, so the Ritz vectors
    agree with the FP64 rotation to FP32 accuracy relative to their size."""
    op = oracle_ops("tiny")
    X = np.random.default_rng(8).standard_normal((op.mesh.ndof, 12))
    Psi_ref, lam_ref = rr.rayleigh_ritz(op, X)
    fe = gpu_fe("tiny", rr_mixed=True)
    Xd = to_dev(X)
    lam = fe.rayleigh_ritz(Xd)
    assert np.abs(lam - lam_ref).max() < 1e-10 * max(1, np.abs(lam_ref).max())
    Psi = Xd.cpu().numpy()
    sgn = np.sign(np.sum(Psi * Psi_ref, 0))
    err = rel_err(Psi * sgn, Psi_ref)
    assert 1e-12 < err < 1e-5, err   # FP32-level, not FP64-level


def test_lanczos_bounds_cover_spectrum():
    """The library's Lanczos runs on Shat^-1 H, the operator that Algorithm 1
    step 2 scales and shifts; its bound must cover that spectrum."""
    op = oracle_ops("tiny")
    Sinv_hat = op.apply_Sinv_approx(np.eye(op.mesh.ndof))
    ev = np.sort(np.linalg.eigvals(Sinv_hat @ op.dense_H()).real)
    fe = gpu_fe("tiny")
    tmin, up = fe.lanczos_bounds(20, 7)
    assert up >= ev[-1] * (1 - 1e-3)
    assert up < 1.3 * ev[-1]
    assert tmin >= ev[0] - 1e-6


def _rchfsi_gpu(fe, X0, m, iters, prec, nwanted):
    import torch
    X = to_dev(X0)
    lam = fe.rayleigh_ritz(X)
    tmin, bU = fe.lanczos_bounds(20, 7)
    out = torch.empty_like(X)
    hist = []
    for _ in range(iters):
        bounds = (min(lam[0], tmin), lam[-1], bU)
        fe.cheb_filter(X, lam, m, bounds, prec=prec, out=out)
        X, out = out, X
        lam = fe.rayleigh_ritz(X)
        hist.append((lam.copy(), fe.residuals(X[:, :nwanted], lam[:nwanted])))
    return X, lam, hist


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16", "tf32-y32", "tf32-rrmix", "tf32-pair"])
def test_rchfsi_converges_to_dense(prec):
    """tiny workload: 10 iterations, degree 20; 8 lowest eigenvalues within 1e-6 Ha of
    the dense FP64 generalised eigensolve of the oracle's matrices ("-y32": the
    residual block Y kept in FP32 only; "-rrmix": mixed-precision subspace rotation;
    "-pair": step 2 in pair-of-FP32 arithmetic)."""
    op = oracle_ops("tiny")
    lam_ex, V_ex = rr.dense_eigs(op, 8)
    y32 = prec.endswith("-y32")
    rrmix = prec.endswith("-rrmix")
    pair = prec.endswith("-pair")
    prec = prec.split("-")[0]
    fe = gpu_fe("tiny", block=16, y0_fp32=y32, rr_mixed=rrmix, y0_pair32=pair)
    X0 = inputs.start_columns("tiny", range(16))
    X, lam, hist = _rchfsi_gpu(fe, X0, 20, 10, prec, 8)
    err = np.abs(lam[:8] - lam_ex).max()
    assert err < 1e-6, (prec, err, [h[0][:8] - lam_ex for h in hist[-2:]])
    # subspace of the 8 lowest states: principal angles in the S inner product
    ang = rr.subspace_angles_S(op.apply_S, X.cpu().numpy()[:, :8], V_ex)
    assert ang.max() < 1e-3
