"""Pins for Rayleigh-Ritz, bounds and the R-ChFSI driver (Algorithm 1)."""
import numpy as np
import pytest

import inputs
from oracle import ops as O
from oracle import rr
from tests.test_oracle_cheb import _tiny_ops


def test_ritz_values_above_eigenvalues():
    """Courant-Fischer: the k-th Ritz value >= the k-th eigenvalue."""
    op = _tiny_ops()
    lam, _ = rr.dense_eigs(op, 10)
    X = np.random.default_rng(3).standard_normal((op.mesh.ndof, 10))
    _, ritz = rr.rayleigh_ritz(op, X)
    assert np.all(ritz >= lam - 1e-10)


def test_lanczos_upper_bound():
    op = _tiny_ops()
    ev = np.linalg.eigvalsh(np.linalg.solve(np.linalg.cholesky(op.dense_S()),
                                            np.linalg.solve(np.linalg.cholesky(op.dense_S()),
                                                            op.dense_H()).T))
    tmin, up = rr.lanczos_bounds(lambda x: op.apply_Sinv_exact(op.apply_H(x)),
                                 op.apply_S, op.mesh.ndof)
    assert up >= ev[-1] - 1e-8
    assert up < 1.2 * ev[-1]
    assert tmin >= ev[0] - 1e-10


@pytest.mark.slow
def test_tiny_workload_converges_to_dense():
    """tiny workload: 10 R-ChFSI iterations, 8 lowest vs dense eigh <= 1e-6 Ha."""
    s = inputs.make_system("tiny")
    op = O.PawOperators(s)
    lam_ex, _ = rr.dense_eigs(op, 8)
    X0 = inputs.start_columns("tiny", range(16))
    hist = []
    Psi, lam, _ = rr.rchfsi(op, X0, 20, 10, 8, sinv="approx", history=hist)
    assert np.abs(lam[:8] - lam_ex).max() < 1e-6
    assert hist[-1][1].max() < 1e-4
