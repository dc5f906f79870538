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


# ---------------------------------------------------------------------------
# Principal angles in the S inner product (the comparison of subspaces in the
# accuracy checks).  Pinned on constructed spans whose angles are known exactly.
# ---------------------------------------------------------------------------
def _spd(n, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * rng.uniform(0.2, 5.0, n)) @ Q.T


def _s_orthonormal(S, k, rng):
    """k vectors q_i with q_i^T S q_j = delta_ij (not Euclidean-orthonormal)."""
    Lc = np.linalg.cholesky(S)
    Z, _ = np.linalg.qr(rng.standard_normal((S.shape[0], k)))
    return np.linalg.solve(Lc.T, Z)


def test_subspace_angles_zero_for_same_span():
    rng = np.random.default_rng(11)
    S = _spd(40, rng)
    U = rng.standard_normal((40, 5))
    V = U @ rng.standard_normal((5, 5))
    ang = rr.subspace_angles_S(lambda A: S @ A, U, V)
    assert ang.shape == (5,)
    assert ang.max() < 1e-12


def test_subspace_angles_right_for_s_orthogonal_spans():
    rng = np.random.default_rng(12)
    S = _spd(40, rng)
    U = rng.standard_normal((40, 4))
    W = rng.standard_normal((40, 4))
    V = W - U @ np.linalg.solve(U.T @ S @ U, U.T @ S @ W)      # S-orthogonal to span(U)
    ang = rr.subspace_angles_S(lambda A: S @ A, U, V)
    np.testing.assert_allclose(ang, np.pi / 2, atol=1e-12)
    # the same spans are not orthogonal in the Euclidean inner product
    eu = rr.subspace_angles_S(lambda A: A, U, V)
    assert eu.min() < np.pi / 2 - 1e-3


@pytest.mark.parametrize("thetas", [(0.2, 0.7, 1.3), (1e-6, 3e-4, 0.05)])
def test_subspace_angles_known(thetas):
    """span(q1, q2, q3) vs span(cos t_i q_i + sin t_i q_{i+3}) with S-orthonormal q has
    principal angles t_i, whatever basis of the second span is passed."""
    rng = np.random.default_rng(13)
    S = _spd(50, rng)
    Q = _s_orthonormal(S, 6, rng)
    U = Q[:, :3] @ rng.standard_normal((3, 3))
    t = np.array(thetas)
    V = (Q[:, :3] * np.cos(t) + Q[:, 3:] * np.sin(t)) @ rng.standard_normal((3, 3))
    ang = np.sort(rr.subspace_angles_S(lambda A: S @ A, U, V))
    np.testing.assert_allclose(ang, np.sort(t), rtol=1e-6, atol=0)
    # with the Euclidean inner product the angles differ (S is not a multiple of I)
    eu = np.sort(rr.subspace_angles_S(lambda A: A, U, V))
    assert np.abs(eu - np.sort(t)).max() > 1e-3


def test_subspace_angles_unequal_dimensions():
    """span(q1) inside span(q1, q2) has the one angle 0, in either order of the arguments;
    span(cos t q1 + sin t q3) against span(q1, q2) has the one angle t."""
    rng = np.random.default_rng(14)
    S = _spd(30, rng)
    Q = _s_orthonormal(S, 3, rng)
    big = Q[:, :2] @ rng.standard_normal((2, 2))
    for a, b in ((Q[:, :1], big), (big, Q[:, :1])):
        ang = rr.subspace_angles_S(lambda A: S @ A, a, b)
        assert ang.shape == (1,) and ang[0] < 1e-12
    v = np.cos(0.4) * Q[:, :1] + np.sin(0.4) * Q[:, 2:3]
    np.testing.assert_allclose(rr.subspace_angles_S(lambda A: S @ A, big, v), [0.4], rtol=1e-12)
