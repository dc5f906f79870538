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
