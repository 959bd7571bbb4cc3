"""Pins of the oracle's Roe-type entropy-stable matrix dissipation.  The pins use properties fixed
by the mathematics and by autograd, not by the formulas themselves:
* dq/dw is the inverse of the autograd Jacobian of the entropy variables;
* D(n) equals |A_n| dq/dw, with |A_n| the matrix absolute value of the autograd flux Jacobian taken
  by eigendecomposition;
* D is symmetric positive semidefinite, so the interface term produces entropy;
* the scheme with it conserves, preserves a freestream, and dissipates less entropy than the local
  Lax-Friedrichs reading on the same state."""
import math

import numpy as np
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I

F64 = torch.float64


def _states(n, seed, gas):
    g = torch.Generator().manual_seed(seed)
    rho = 0.5 + torch.rand(n, generator=g, dtype=F64)
    u = torch.randn(3, n, generator=g, dtype=F64)
    p = gas.R * (0.5 + torch.rand(n, generator=g, dtype=F64))
    E = p / (gas.gamma - 1.0) + 0.5 * rho * (u ** 2).sum(0)
    return torch.stack([rho, rho * u[0], rho * u[1], rho * u[2], E], dim=1)


def test_dq_dw_is_the_inverse_entropy_hessian():
    gas = O.Gas.from_mach(0.3, 0.0)
    q = _states(8, 1, gas)
    rho, u, p, _ = O.primitives(q, gas)
    M = O.dq_dw(rho, u, p, gas)
    for i in range(q.shape[0]):
        Jw = torch.autograd.functional.jacobian(lambda x: O.entropy_variables(x[None], gas)[0], q[i])
        assert torch.allclose(M[i] @ Jw, torch.eye(5, dtype=F64), atol=1e-11)
        assert torch.allclose(M[i], M[i].T, atol=1e-12)


def test_matrix_dissipation_is_abs_flux_jacobian_times_dq_dw():
    gas = O.Gas.from_mach(0.3, 0.0)
    q = _states(6, 2, gas)
    rho, u, p, _ = O.primitives(q, gas)
    g = torch.Generator().manual_seed(3)
    n = [torch.randn(6, generator=g, dtype=F64) * 2.0 for _ in range(3)]
    D = O.matrix_dissipation(rho, u, p, n, gas)
    M = O.dq_dw(rho, u, p, gas)
    for i in range(6):
        ni = [n[d][i:i + 1] for d in range(3)]
        A = torch.autograd.functional.jacobian(lambda x: O.euler_flux_n(x[None], ni, gas)[0], q[i]).numpy()
        lam, V = np.linalg.eig(A)
        absA = (V @ np.diag(np.abs(lam)) @ np.linalg.inv(V)).real
        want = absA @ M[i].numpy()
        assert np.allclose(D[i].numpy(), want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
        ev = np.linalg.eigvalsh(0.5 * (D[i].numpy() + D[i].numpy().T))
        assert ev.min() >= -1e-12 * ev.max()
        assert np.allclose(D[i].numpy(), D[i].numpy().T, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def _mesh(p, k, warp, seed):
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), *k, [-math.pi] * 3, [math.pi] * 3, warp=warp, seed=seed)
    return O.make_mesh(p, x, *k), x


def test_matrix_dissipation_scheme_conserves_preserves_freestream_and_produces_less_entropy():
    gas = O.Gas.from_mach(0.3, 0.0)
    mesh, x = _mesh(3, (3, 2, 2), 0.1, 7)
    qf = torch.tensor(I.freestream(x, Ma=0.3))
    assert float(O.rhs(qf, mesh, gas, dissipation="matrix").abs().max()) < 1e-11 * gas.R
    q = torch.tensor(I.perturb(I.taylor_green(x, Ma=0.3), seed=4, rel=0.05))
    PJ = O.quadrature_weights(mesh)
    r = O.rhs(q, mesh, gas, dissipation="matrix")
    for v in range(5):
        assert abs(float((PJ * r[:, v]).sum())) <= 1e-12 * float((PJ * r[:, v].abs()).sum())
    _, _, dS_m, _ = O.budgets(q, r, mesh, gas)
    _, _, dS_l, _ = O.budgets(q, O.rhs(q, mesh, gas, dissipation=True), mesh, gas)
    _, _, dS_0, _ = O.budgets(q, O.rhs(q, mesh, gas, dissipation=False), mesh, gas)
    scale = float((PJ * (O.entropy_variables(q, gas) * r).sum(dim=1).abs()).sum())
    assert abs(dS_0) <= 1e-12 * scale
    assert dS_l < dS_m < -1e-8 * scale


def test_interior_penalty_conserves_produces_entropy_and_is_linear():
    """The interior-penalty term: global conservation, entropy production (dq/dw is positive
    definite and the term is symmetric in the two sides), linearity in its coefficient, no effect on
    a freestream, and no term without viscosity."""
    gas = O.Gas.from_mach(0.3, 200.0)
    mesh, x = _mesh(3, (3, 2, 2), 0.1, 4)
    q = torch.tensor(I.perturb(I.taylor_green(x, Ma=0.3), seed=2, rel=0.05))
    r0 = O.rhs(q, mesh, gas)
    d1 = O.rhs(q, mesh, gas, ip_coef=1.0) - r0
    d3 = O.rhs(q, mesh, gas, ip_coef=3.0) - r0
    PJ = O.quadrature_weights(mesh)
    for v in range(5):
        assert abs(float((PJ * d1[:, v]).sum())) <= 1e-12 * (float((PJ * d1[:, v].abs()).sum()) + 1e-300)
    assert torch.allclose(d3, 3.0 * d1, rtol=1e-9, atol=1e-12 * float(d1.abs().max()))
    w = O.entropy_variables(q, gas)
    assert float((PJ * (w * d1).sum(dim=1)).sum()) < 0.0
    qf = torch.tensor(I.freestream(x, Ma=0.3))
    assert float((O.rhs(qf, mesh, gas, ip_coef=2.0) - O.rhs(qf, mesh, gas)).abs().max()) == 0.0
    inv = O.Gas.from_mach(0.3, 0.0)
    assert torch.equal(O.rhs(q, mesh, inv, ip_coef=2.0), O.rhs(q, mesh, inv))
