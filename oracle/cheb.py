"""Chebyshev filtering for the oracle (FP64).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

* ``chebyshev_T``      closed form of T_m (cos / cosh), Eq. ChFSI recurrance.
* ``scaled_scalar``    C_m(x) = T_m(x~) / T_m(a0~) for scalars.
* ``classical_filter`` Eq. ChFSI recurrance2: X_{t+1} = (2 z_{t+1}/e) S^-1 H X_t
                       - (2 z_{t+1} c / e) X_t - z_t z_{t+1} X_{t-1}.
* ``rchfsi_filter``    Algorithm 2 (residual-based Chebyshev filtered subspace),
                       taken step by step with an arbitrary S^-1 (exact or the
                       approximate inverse of Eq. Sinvapprox).

Degree convention (the equations iterate one step further than Algorithm 2's
loop): Algorithm 2 is authoritative.  A filter of degree m applies H once in
its step 2 and m-1 times in its loop, and returns C_m.
"""
from __future__ import annotations

import numpy as np


def chebyshev_T(m: int, x):
    """T_m(x) from its closed form: cos(m acos x) on [-1, 1], cosh outside."""
    x = np.asarray(x, float)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    hi = x > 1.0
    out[hi] = np.cosh(m * np.arccosh(x[hi]))
    lo = x < -1.0
    out[lo] = (-1.0) ** m * np.cosh(m * np.arccosh(-x[lo]))
    return out


def filter_constants(a0: float, bW: float, bU: float):
    """e, c and zeta_1 of Algorithm 2 step 1."""
    e = (bU - bW) / 2.0
    c = (bU + bW) / 2.0
    return e, c, e / (a0 - c)


def scaled_scalar(m: int, lam, a0: float, bW: float, bU: float):
    """C_m(lambda~, a0~) = T_m((lam-c)/e) / T_m((a0-c)/e) via the closed form."""
    e, c, _ = filter_constants(a0, bW, bU)
    lam = np.asarray(lam, float)
    return chebyshev_T(m, (lam - c) / e) / chebyshev_T(m, np.array([(a0 - c) / e]))[0]


def classical_filter(apply_SinvH, X, m: int, a0: float, bW: float, bU: float):
    """Scaled classical filter C_m(S^-1 H) X by Eq. ChFSI recurrance2."""
    e, c, z1 = filter_constants(a0, bW, bU)
    X0 = np.array(X, float)
    X1 = (z1 / e) * (apply_SinvH(X0) - c * X0)
    zeta = z1
    for _t in range(1, m):
        znew = 1.0 / (2.0 / z1 - zeta)
        X2 = (2 * znew / e) * apply_SinvH(X1) - (2 * znew * c / e) * X1 - zeta * znew * X0
        X0, X1 = X1, X2
        zeta = znew
    return X1 if m >= 1 else X0


def rchfsi_filter(apply_H, apply_S, apply_Sinv, X, lam, m: int,
                  a0: float, bW: float, bU: float, trace=None):
    """Algorithm 2, steps 1-5, in the paper's order and notation.

    X: (ndof, B) block Psi_in (real, or complex for the problem at a Bloch
    wavevector k); lam: (B,) eigenvalue estimates Lambda (real: H, S are
    Hermitian).  Returns Psi_f = S^-1 R_Y + X Lambda_Y.  ``trace`` (a list)
    receives the per-iteration (zeta, Lambda_Y) after each loop step.
    """
    X = np.asarray(X)
    X = X if np.iscomplexobj(X) else X.astype(float)
    lam = np.asarray(lam, float)
    # step 1
    e = (bU - bW) / 2.0
    c = (bU + bW) / 2.0
    zeta = e / (a0 - c)
    zeta1 = zeta
    gamma = 2.0 / zeta1
    # step 2
    Y = apply_H(X) - apply_S(X) * lam[None, :]
    # step 3
    RX = np.zeros_like(X)
    RY = (zeta1 / e) * Y
    LX = np.ones_like(lam)
    LY = (zeta1 / e) * (lam - c)
    # step 4
    for _theta in range(2, m + 1):
        zeta1 = 1.0 / (gamma - zeta)
        RX = ((2 * zeta1 / e) * apply_H(apply_Sinv(RY)) - (2 * zeta1 / e) * c * RY
              - zeta * zeta1 * RX + (2 * zeta1 / e) * Y * LY[None, :])
        LX = (2 * zeta1 / e) * LY * lam - (2 * zeta1 / e) * c * LY - zeta * zeta1 * LX
        RX, RY = RY, RX
        LX, LY = LY, LX
        zeta = zeta1
        if trace is not None:
            trace.append((zeta, LY.copy()))
    # step 5
    return apply_Sinv(RY) + X * LY[None, :]


def recurrence_scalars(m: int, a0: float, bW: float, bU: float):
    """(alpha, beta, gamma) of Eq. HXCheby for loop steps theta = 2..m.

    alpha = 2 z_t / e, beta = 2 z_t c / e, gamma = z_{t-1} z_t (signs absorbed).
    """
    e = (bU - bW) / 2.0
    c = (bU + bW) / 2.0
    z1 = e / (a0 - c)
    zeta = z1
    out = []
    for _t in range(2, m + 1):
        zn = 1.0 / (2.0 / z1 - zeta)
        out.append((2 * zn / e, 2 * zn * c / e, zeta * zn))
        zeta = zn
    return out


def chebyshev_growth(m: int, a0: float, bW: float, bU: float) -> float:
    """|T_m(a0~)|, the amplification of the lowest wanted state."""
    e, c, _ = filter_constants(a0, bW, bU)
    return float(abs(chebyshev_T(m, np.array([(a0 - c) / e]))[0]))
