"""Accuracy of the mixed-precision filter at the full size of the mid workload.

The throughput figure of the mixed (TF32) filter is quoted at converged eigenvalue error
<= 1e-6 Ha and subspace angles <= 1e-5.  At 884,736 DoFs no dense solve exists, so the
reference is the same R-ChFSI iteration (Algorithm 1 with Algorithm 2 as the filter, FP64
Rayleigh-Ritz) with the FP64 filter, whose operators and filter output match the FP64 oracle
at this size (test_gpu_fullsize.py).  Both arms start from the same S-orthonormal Ritz
vectors of a seeded random block (512 vectors in blocks of 256, Chebyshev degree 30) and run
the same number of iterations.  Compared: the lowest k = 256 states (moved to the nearest
index with a gap above 1e-4 Ha, so no degenerate level is split): eigenvalues, principal
angles in the S inner product (the oracle's pinned checker, with the library's FP64 S), and
the FP64 residual norms of both arms as the evidence of convergence.
"""
import numpy as np
import pytest

import inputs
from oracle import rr
from tests.gpu_util import gap_index, report

pytestmark = pytest.mark.gpu

ITERS = 16


def _rchfsi(fe, X0, lam0, tmin, bU, m, prec, iters):
    import torch
    X = X0.clone()
    lam = lam0.copy()
    out = torch.empty_like(X)
    for _ in range(iters):
        fe.cheb_filter(X, lam, m, (min(lam[0], tmin), float(lam[-1]), bU), prec=prec, out=out)
        X, out = out, X
        lam = fe.rayleigh_ritz(X)
        fe.sync_status()
    del out
    return X, lam, fe.residuals(X, lam)


def test_mixed_filter_matches_fp64_at_mid():
    import torch
    import paper_2604_26037_gb300 as P
    cfg = inputs.CONFIGS["mid"]
    fe = P.PawFE.from_system(inputs.make_system("mid"), block=cfg["block"])
    g = torch.Generator(device="cuda").manual_seed(1234)
    X0 = torch.randn((fe.ndof, cfg["nvec"]), dtype=torch.float64, device="cuda", generator=g)
    lam0 = fe.rayleigh_ritz(X0)
    tmin, bU = fe.lanczos_bounds(20, 7)
    Xa, la, ra = _rchfsi(fe, X0, lam0, tmin, bU, cfg["degree"], "tf32", ITERS)
    Xb, lb, rb = _rchfsi(fe, X0, lam0, tmin, bU, cfg["degree"], "fp64", ITERS)
    del X0
    k = gap_index(lb, cfg["nvec"] // 2)
    dlam = np.abs(la[:k] - lb[:k]).max()

    def S_apply(A):
        return fe.apply_S(torch.from_numpy(np.ascontiguousarray(A)).cuda()).cpu().numpy()

    ang = rr.subspace_angles_S(S_apply, Xa[:, :k].cpu().numpy(), Xb[:, :k].cpu().numpy())
    name = f"mid R-ChFSI tf32 vs fp64, {ITERS} iterations, lowest {k}"
    report(name, "max |eigenvalue difference| (Ha)", dlam, 1e-6)
    report(name, "max principal angle (S inner product)", ang.max(), 1e-5)
    report(name, "max residual tf32", ra[:k].max(), 1e-5)
    report(name, "max residual fp64", rb[:k].max(), 1e-5)
    fe.close()
    assert k >= 200
    assert ra[:k].max() < 1e-5 and rb[:k].max() < 1e-5     # both arms converged on these states
    assert dlam <= 1e-6
    assert ang.max() <= 1e-5
