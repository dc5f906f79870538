"""Pins for the energy gradient: E = tr(X^T H X) is linear in V and Delta_H,
so central finite differences are exact up to rounding."""
import numpy as np

from oracle import grad
from oracle import ops as O
from tests.test_oracle_cheb import _tiny_ops


def test_grad_V_and_D_by_finite_differences():
    op = _tiny_ops()
    rng = np.random.default_rng(9)
    X = rng.standard_normal((op.mesh.ndof, 3))
    dV, dD = grad.energy_grad(op, X)
    s = op.sysd
    dirV = rng.standard_normal(op.Vq.shape)
    dirD = rng.standard_normal(op.D.shape)
    h = 1e-4
    Ep = grad.energy(O.PawOperators(s, Vq=op.Vq + h * dirV), X)
    Em = grad.energy(O.PawOperators(s, Vq=op.Vq - h * dirV), X)
    fd = (Ep - Em) / (2 * h)
    assert abs(fd - np.sum(dV * dirV)) < 1e-6 * abs(fd)
    Ep = grad.energy(O.PawOperators(s, D=op.D + h * dirD), X)
    Em = grad.energy(O.PawOperators(s, D=op.D - h * dirD), X)
    fd = (Ep - Em) / (2 * h)
    assert abs(fd - np.sum(dD * dirD)) < 1e-6 * abs(fd)


def test_density_pins():
    """rho and D^a of Eq. FE PAW governing equations (Gamma point, one spin):
    the integral of rho equals sum_i f_i x_i^T M x_i with the separately assembled
    consistent mass matrix (both quadratures are exact for products of degree-p
    functions); with unit occupations rho w_q detJ and D^a are the energy gradient
    (pinned above by finite differences); D^a is symmetric positive semidefinite."""
    op = _tiny_ops()
    rng = np.random.default_rng(10)
    X = rng.standard_normal((op.mesh.ndof, 5))
    f = rng.uniform(0.0, 2.0, 5)
    rho, D = grad.density(op, X, f)
    total = np.sum(op.Wq[None, :] * rho)
    ref = np.sum(f * np.sum(X * op.apply_M(X), axis=0))
    assert abs(total - ref) < 1e-12 * abs(ref)
    rho1, D1 = grad.density(op, X)
    dV, dD = grad.energy_grad(op, X)
    assert np.abs(op.Wq[None, :] * rho1 - dV).max() < 1e-13 * np.abs(dV).max()
    assert np.abs(D1 - dD).max() < 1e-13 * np.abs(dD).max()
    for a in range(op.natoms):
        assert np.abs(D[a] - D[a].T).max() < 1e-14 * np.abs(D[a]).max()
        assert np.linalg.eigvalsh(D[a]).min() > -1e-12 * np.abs(D[a]).max()


def test_hellmann_feynman_at_eigenvectors():
    """S depends on neither V nor Delta_H, so at S-orthonormal eigenvectors X of
    H x = lambda S x the derivative of the sum of the lowest k eigenvalues along a direction
    of V (or of Delta_H) is the gradient of E = tr(X^T H X) at X contracted with that
    direction (k taken at a gap, where the sum is smooth)."""
    import scipy.linalg as sla
    from tests.test_oracle_ops import _two_atom
    s = _two_atom()
    op = O.PawOperators(s)
    w, V = sla.eigh(op.dense_H(), op.dense_S())
    k = next(j for j in range(6, 40) if w[j] - w[j - 1] > 1e-2)
    dV, dD = grad.energy_grad(op, V[:, :k])
    rng = np.random.default_rng(12)
    dirV = rng.standard_normal(op.Vq.shape)
    dirD = rng.standard_normal(op.D.shape)
    dirD = 0.5 * (dirD + np.transpose(dirD, (0, 2, 1)))   # symmetric, as Delta_H
    h = 1e-5

    def lowest(**kw):
        o = O.PawOperators(s, **kw)
        return np.sum(sla.eigh(o.dense_H(), o.dense_S(), eigvals_only=True)[:k])

    fd = (lowest(Vq=op.Vq + h * dirV) - lowest(Vq=op.Vq - h * dirV)) / (2 * h)
    assert abs(fd - np.sum(dV * dirV)) < 1e-6 * abs(fd)
    fd = (lowest(D=op.D + h * dirD) - lowest(D=op.D - h * dirD)) / (2 * h)
    assert abs(fd - np.sum(dD * dirD)) < 1e-6 * abs(fd)
