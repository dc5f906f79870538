"""GPU parity at a Bloch wavevector k (complex multivectors) against the k-point oracle.

Operators H(k), S(k), Shat^-1(k) in FP64 / FP32 / TF32 on three meshes (p = 4, 5, 6;
4, 9 and 13 projectors, i.e. both stored-projector paddings), ragged and aligned
column counts; Algorithm 2 at k; complex Rayleigh-Ritz and residual norms; the
Lanczos bound on Shat^-1 H; R-ChFSI at k converging to the dense eigensolve.
"""
import functools

import numpy as np
import pytest

from oracle import cheb, kpoint, rr
from tests.gpu_util import gpu_fe, system, to_dev

pytestmark = pytest.mark.gpu

KVEC = {"tiny": (0.11, -0.07, 0.05), "p5": (-0.2, 0.1, 0.15), "p6": (0.09, 0.13, -0.06)}


@functools.lru_cache(maxsize=None)
def kops(name):
    return kpoint.PawOperatorsK(system(name), KVEC[name])


def cvec(n, ncols, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))


def crel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@functools.lru_cache(maxsize=None)
def kfe(name):
    return gpu_fe(name, kpoint=KVEC[name])


@pytest.mark.parametrize("name", ["tiny", "p5", "p6"])
@pytest.mark.parametrize("ncols", [37, 64])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5), ("tf32", 4e-3), ("bf16", 3e-2)])
def test_operators_at_k(name, ncols, prec, tol):
    import torch
    op, fe = kops(name), kfe(name)
    assert fe.complex
    X = cvec(op.mesh.ndof, ncols, 11)
    if prec != "fp64":
        X = X.astype(np.complex64).astype(np.complex128)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    Xd = to_dev(X, dt)
    for fn, ref in ((fe.apply_H, op.apply_H), (fe.apply_S, op.apply_S),
                    (fe.apply_Sinv_approx, op.apply_Sinv_approx)):
        Y = fn(Xd, prec=prec).cpu().numpy().astype(np.complex128)
        assert crel(Y, ref(X)) < tol, fn.__name__


def test_k0_handle_stays_real():
    fe = gpu_fe("tiny", kpoint=(0.0, 0.0, 0.0))
    assert not fe.complex


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("tf32", 2e-2), ("bf16", 1e-1)])
def test_filter_at_k(prec, tol):
    op, fe = kops("tiny"), kfe("tiny")
    X = cvec(op.mesh.ndof, 20, 12)
    lam = np.linspace(-0.4, 0.3, 20)
    bounds = (-0.6, 0.35, 95.0)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, X, lam, 6, *bounds)
    out = fe.cheb_filter(to_dev(X), lam, 6, bounds, prec=prec).cpu().numpy()
    assert crel(out, ref) < tol


def test_filter_at_k_in_blocks_with_a_ragged_tail():
    """block width 8 over 21 complex columns (blocks 8, 8, 5) against the single-call oracle"""
    import paper_2604_26037_gb300 as P
    op = kops("tiny")
    fe = P.PawFE.from_system(system("tiny"), kpoint=KVEC["tiny"], block=8)
    X = cvec(op.mesh.ndof, 21, 15)
    lam = np.linspace(-0.4, 0.3, 21)
    bounds = (-0.6, 0.35, 95.0)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, X, lam, 5, *bounds)
    out = fe.cheb_filter(to_dev(X), lam, 5, bounds, prec="fp64").cpu().numpy()
    assert crel(out, ref) < 1e-10
    fe.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("tf32", 2e-2)])
def test_filter_at_k_overlapped_blocks(prec, tol):
    """21 complex columns in blocks of 8 (8, 8, 5): by default step 2 of each next block runs
    beside the loop of the current one on the handle's two streams; it matches the
    one-after-another schedule and the oracle."""
    import paper_2604_26037_gb300 as P
    op = kops("tiny")
    fe_o = P.PawFE.from_system(system("tiny"), kpoint=KVEC["tiny"], block=8)
    fe_s = P.PawFE.from_system(system("tiny"), kpoint=KVEC["tiny"], block=8, overlap=False)
    X = cvec(op.mesh.ndof, 21, 16)
    lam = np.linspace(-0.4, 0.3, 21)
    bounds = (-0.6, 0.35, 95.0)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, X, lam, 5, *bounds)
    Xd = to_dev(X)
    o = fe_o.cheb_filter(Xd, lam, 5, bounds, prec=prec).cpu().numpy()
    s_ = fe_s.cheb_filter(Xd, lam, 5, bounds, prec=prec).cpu().numpy()
    fe_o.sync_status()
    assert crel(o, ref) < tol and crel(s_, ref) < tol
    assert crel(o, s_) < (1e-5 if prec == "fp32" else 4e-3)
    fe_o.close()
    fe_s.close()


def test_rayleigh_ritz_and_residuals_at_k():
    import torch
    op, fe = kops("tiny"), kfe("tiny")
    X = cvec(op.mesh.ndof, 12, 13)
    Psi_ref, lam_ref = rr.rayleigh_ritz(op, X)
    Xd = to_dev(X)
    lam = fe.rayleigh_ritz(Xd)
    assert np.max(np.abs(lam - lam_ref)) < 1e-10 * max(1.0, np.max(np.abs(lam_ref)))
    Psi = Xd.cpu().numpy()
    G = Psi.conj().T @ op.apply_S(Psi)
    assert np.max(np.abs(G - np.eye(12))) < 1e-10
    r = fe.residuals(Xd, lam)
    r_ref = rr.residual_norms(op, Psi, lam)
    assert np.max(np.abs(r - r_ref)) < 1e-9 * max(1.0, np.max(r_ref))
    assert Xd.dtype == torch.complex128


@functools.lru_cache(maxsize=None)
def tiny3():
    """the tiny workload on 3^3 cells of degree 3 (729 DoFs): small enough for dense solves"""
    return dict(system("tiny"), ncell=3, p=3)


def test_lanczos_bounds_at_k():
    """The bound of the library's Lanczos covers the spectrum of Shat^-1 H at k."""
    import paper_2604_26037_gb300 as P
    op = kpoint.PawOperatorsK(tiny3(), KVEC["tiny"])
    fe = P.PawFE.from_system(tiny3(), kpoint=KVEC["tiny"])
    n = op.mesh.ndof
    Sinv_hat = op.apply_Sinv_approx(np.eye(n))
    ev = np.sort(np.linalg.eigvals(Sinv_hat @ op.dense_H()).real)
    tmin, up = fe.lanczos_bounds(20, 7)
    assert up >= ev[-1] * (1 - 1e-3)
    assert up < 1.3 * ev[-1]
    assert tmin >= ev[0] - 1e-6
    fe.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_rchfsi_at_k_converges_to_dense(prec):
    import torch

    import paper_2604_26037_gb300 as P
    sysd = tiny3()
    k = KVEC["tiny"]
    op = kpoint.PawOperatorsK(sysd, k)
    exact, _ = op.dense_eigs(8)
    fe = P.PawFE.from_system(sysd, kpoint=k, block=16)
    X = to_dev(cvec(op.mesh.ndof, 12, 14))
    lam = fe.rayleigh_ritz(X)
    tmin, bU = fe.lanczos_bounds(20, 7)
    out = torch.empty_like(X)
    for _ in range(12):
        fe.cheb_filter(X, lam, 16, (min(lam[0], tmin), lam[-1], bU), prec=prec, out=out)
        X, out = out, X
        lam = fe.rayleigh_ritz(X)
    assert np.max(np.abs(lam[:8] - exact)) < 1e-6
    r = fe.residuals(X[:, :8], lam[:8])
    assert np.max(r) < 1e-4
    fe.close()
