"""Pins for the oracle's Chebyshev filters (Eqs. ChFSI recurrance/2,
Eqs. RChFSI residual 0/1, RChFSI final, Algorithm 2)."""
import numpy as np
from numpy.polynomial import chebyshev as npcheb

from oracle import cheb
from oracle import ops as O
from oracle import rr
from tests.oracle_systems import mini_system, sym_random


def test_chebyshev_closed_form():
    x = np.linspace(-3.0, 3.0, 41)
    for m in range(0, 12):
        c = np.zeros(m + 1)
        c[m] = 1.0
        np.testing.assert_allclose(cheb.chebyshev_T(m, x), npcheb.chebval(x, c),
                                   rtol=1e-11, atol=1e-11)


def test_zeta_ratios():
    """zeta_t = T_{t-1}(a0~)/T_t(a0~): the scalars of Eq. HXCheby."""
    a0, bW, bU = -0.7, 0.4, 9.0
    e, c, _ = cheb.filter_constants(a0, bW, bU)
    t0 = (a0 - c) / e
    sc = cheb.recurrence_scalars(12, a0, bW, bU)
    for k, (al, be, ga) in enumerate(sc):
        t = k + 2
        Tm1, T, Tm2 = (cheb.chebyshev_T(t - 1, np.array([t0]))[0],
                       cheb.chebyshev_T(t, np.array([t0]))[0],
                       cheb.chebyshev_T(t - 2, np.array([t0]))[0])
        zt = Tm1 / T
        zprev = Tm2 / Tm1
        assert abs(al - 2 * zt / e) < 1e-13 * abs(al)
        assert abs(be - 2 * zt * c / e) < 1e-13 * abs(be)
        assert abs(ga - zprev * zt) < 1e-13 * abs(ga)


def _diag_ops(lam_diag):
    d = np.asarray(lam_diag, float)
    H = lambda X: d[:, None] * X
    S = lambda X: np.array(X, float)
    return H, S


def test_classical_filter_diagonal():
    rng = np.random.default_rng(0)
    d = np.sort(rng.uniform(-1.0, 20.0, 40))
    H, S = _diag_ops(d)
    x = rng.standard_normal((40, 2))
    a0, bW, bU = d[0] - 0.1, d[9], 20.5
    for m in (1, 2, 7, 15):
        out = cheb.classical_filter(H, x, m, a0, bW, bU)
        ref = cheb.scaled_scalar(m, d, a0, bW, bU)[:, None] * x
        np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-12)


def test_rchfsi_diagonal_closed_form():
    """Algorithm 2 with diagonal H, S = I, exact inverse: C_m(lambda~) x."""
    rng = np.random.default_rng(1)
    d = np.sort(rng.uniform(-1.0, 20.0, 30))
    H, S = _diag_ops(d)
    x = rng.standard_normal((30, 3))
    lam = rng.uniform(0, 5, 3)
    a0, bW, bU = d[0] - 0.1, d[8], 20.5
    for m in (2, 5, 20):
        out = cheb.rchfsi_filter(H, S, S, x, lam, m, a0, bW, bU)
        ref = cheb.scaled_scalar(m, d, a0, bW, bU)[:, None] * x
        np.testing.assert_allclose(out, ref, rtol=1e-9, atol=1e-9)


def _tiny_ops():
    rng = np.random.default_rng(11)
    s = mini_system(L=10.0, n=2, p=4, positions=[[2.1, 3.7, 4.9], [6.2, 5.1, 3.3]],
                    D=sym_random(rng, 2, 4, 0.1), dS=sym_random(rng, 2, 4, 0.02),
                    vdepth=2.0, vwidth=1.0)
    return O.PawOperators(s)


def test_rchfsi_equals_classical_with_exact_inverse():
    """The residual recurrence is algebraically the classical filter."""
    op = _tiny_ops()
    rng = np.random.default_rng(2)
    X = rng.standard_normal((op.mesh.ndof, 4))
    lam = np.array([-0.4, 0.1, 0.3, 0.5])
    a0, bW, bU = -0.6, 0.8, 95.0
    m = 12
    SinvH = lambda Z: op.apply_Sinv_exact(op.apply_H(Z))
    ref = cheb.classical_filter(SinvH, X, m, a0, bW, bU)
    out = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_exact, X, lam, m, a0, bW, bU)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_rchfsi_fixed_point_any_inverse():
    """Exact eigenpairs in: R_1 = 0, so Psi_f = Psi C_m(Lambda~) for any S^-1."""
    op = _tiny_ops()
    lam, V = rr.dense_eigs(op, 6)
    a0, bW, bU = lam[0] - 0.05, lam[-1], 95.0
    out = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, V, lam, 20, a0, bW, bU)
    ref = V * cheb.scaled_scalar(20, lam, a0, bW, bU)[None, :]
    np.testing.assert_allclose(out, ref, atol=1e-8 * np.abs(ref).max())
