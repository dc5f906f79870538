"""GPU parity: energy tr(X^T H X) and its adjoint (gradient with respect to V at
the quadrature points and to Delta_H), against the oracle gradient and
central finite differences through the autograd Function."""
import numpy as np
import pytest

from oracle import grad as G
from tests.gpu_util import gpu_fe, oracle_ops, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_energy_and_gradient_vs_oracle(prec):
    import torch
    op = oracle_ops("tiny")
    X = np.random.default_rng(12).standard_normal((op.mesh.ndof, 6))
    fe = gpu_fe("tiny")
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = to_dev(X, dt)
    Xr = Xd.double().cpu().numpy()
    E = fe.energy(Xd, prec)
    assert abs(E - G.energy(op, Xr)) < (1e-11 if prec == "fp64" else 1e-5) * abs(E)
    dV, dD = fe.energy_grad(Xd, prec)
    rV, rD = G.energy_grad(op, Xr)
    assert np.linalg.norm(dV.cpu().numpy() - rV) < 1e-10 * np.linalg.norm(rV)
    assert np.linalg.norm(dD.cpu().numpy() - rD) < (1e-10 if prec == "fp64" else 1e-5) * np.linalg.norm(rD)


def test_autograd_function_matches_finite_differences():
    import torch
    import paper_2604_26037_gb300 as P
    op = oracle_ops("tiny")
    fe = gpu_fe("tiny")
    X = to_dev(np.random.default_rng(13).standard_normal((op.mesh.ndof, 4)))
    Vq = to_dev(op.Vq).requires_grad_(True)
    D = torch.tensor(op.D, dtype=torch.float64, requires_grad=True)
    E = P.SubspaceEnergy.apply(Vq, D, X, fe, "fp64")
    E.backward()
    rng = np.random.default_rng(14)
    dirV = to_dev(rng.standard_normal(op.Vq.shape))
    dirD = rng.standard_normal(op.D.shape)
    dirD = torch.tensor(0.5 * (dirD + dirD.transpose(0, 2, 1)))
    h = 1e-4
    with torch.no_grad():
        Ep = P.SubspaceEnergy.apply(Vq + h * dirV, D, X, fe, "fp64")
        Em = P.SubspaceEnergy.apply(Vq - h * dirV, D, X, fe, "fp64")
        fdV = (Ep - Em).item() / (2 * h)
        Ep = P.SubspaceEnergy.apply(Vq, D + h * dirD, X, fe, "fp64")
        Em = P.SubspaceEnergy.apply(Vq, D - h * dirD, X, fe, "fp64")
        fdD = (Ep - Em).item() / (2 * h)
    gV = torch.sum(Vq.grad * dirV).item()
    gD = torch.sum(D.grad * dirD).item()
    assert abs(fdV - gV) < 1e-5 * abs(gV)
    assert abs(fdD - gD) < 1e-5 * abs(gD)
    fe.set_veff(to_dev(op.Vq))
    fe.set_dij(op.D)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["tiny", "p6"])
def test_density_vs_oracle(prec, name):
    """paw_density: rho at the Gauss points and D^a with random occupations (p6: 13
    projectors stored in the library's internal order, returned in the caller's)."""
    import torch
    op = oracle_ops(name)
    rng = np.random.default_rng(13)
    X = rng.standard_normal((op.mesh.ndof, 7))
    f = rng.uniform(0.0, 2.0, 7)
    fe = gpu_fe(name)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = to_dev(X, dt)
    Xr = Xd.double().cpu().numpy()
    rho, D = fe.density(Xd, f, prec)
    rr, rD = G.density(op, Xr, f)
    tol = 1e-11 if prec == "fp64" else 1e-5
    assert rel_err(rho.cpu().numpy(), rr) < 1e-11   # accumulated in FP64 from the (exact) FP32 inputs
    assert np.linalg.norm(D.cpu().numpy() - rD) < tol * np.linalg.norm(rD)
