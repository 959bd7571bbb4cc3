"""Pins of the oracle's Dormand-Prince integrator (Sec. 5) and of its vector-Jacobian products."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I


def test_dp5_tableau_order_conditions():
    """Row sums equal c, and the 5th-order weights meet the order conditions up to order 5 that
    involve only b and c (quadrature conditions) plus sum b_i a_ij c_j = 1/6."""
    A = [[Fr(v).limit_denominator(10 ** 7) for v in row] for row in O.DP5_A]
    b = [Fr(v).limit_denominator(10 ** 7) for v in O.DP5_B]
    c = [Fr(v).limit_denominator(10 ** 7) for v in O.DP5_C]
    for i, row in enumerate(A):
        assert sum(row, Fr(0)) == c[i]
    for k in range(1, 6):
        assert sum(bi * ci ** (k - 1) for bi, ci in zip(b, c)) == Fr(1, k)
    assert sum(b[i] * sum(A[i][j] * c[j] for j in range(i)) for i in range(6)) == Fr(1, 6)


@pytest.mark.parametrize("f,exact", [
    (lambda y: y, math.e),                 # y' = y, y(0) = 1
    (lambda y: y * y, 1.0 / (1.0 - 0.5)),  # y' = y^2, y(0) = 1, integrated to t = 0.5
])
def test_dp5_fifth_order_convergence(f, exact):
    T = 1.0 if exact == math.e else 0.5
    errs = []
    for n in (8, 64):
        y = O.rk_step(torch.tensor([1.0], dtype=torch.float64), f, T / n, n)
        errs.append(abs(float(y[0]) - exact))
    rate = math.log2(errs[0] / errs[1]) / 3.0      # mean rate over three halvings of dt
    assert rate > 4.7, (errs, rate)


def _small_problem(p=2, k=2, warp=0.1, Re=100.0):
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, [-math.pi] * 3, [math.pi] * 3, warp=warp, seed=1)
    mesh = O.make_mesh(p, x, k, k, k)
    gas = O.Gas.from_mach(0.3, Re)
    q = torch.tensor(I.perturb(I.taylor_green(x, Ma=0.3), seed=4, rel=1e-2))
    return mesh, gas, q


def test_oracle_vjp_matches_central_differences():
    """<v, J u> by central differences of the residual equals <J^T v, u> from the oracle's autograd
    (which uses the log-mean backward pinned against mpmath)."""
    mesh, gas, q = _small_problem()
    g = torch.Generator().manual_seed(1234)
    u = torch.randn(q.shape, generator=g, dtype=torch.float64) * q.abs().amax(dim=(0, 2, 3, 4), keepdim=True)
    v = torch.randn(q.shape, generator=g, dtype=torch.float64)
    qq = q.clone().requires_grad_(True)
    r = O.rhs(qq, mesh, gas)
    (vjp,) = torch.autograd.grad(r, qq, v)
    h = 1e-6
    jvp = (O.rhs(q + h * u, mesh, gas) - O.rhs(q - h * u, mesh, gas)) / (2 * h)
    a, b = float((v * jvp).sum()), float((vjp * u).sum())
    assert abs(a - b) < 1e-6 * abs(b)


def test_oracle_trajectory_gradient_matches_central_differences():
    """d KE(q_n)/d q_0 and d KE/d mu through two DP5 steps: autograd vs central differences."""
    mesh, gas, q0 = _small_problem(p=2, k=2)
    dt = 0.2 * O.cfl_dt(q0, mesh, gas)

    def ke_after(q, mu):
        g2 = O.Gas(gas.gamma, gas.R, mu, gas.Pr)
        qn = O.rk_step(q, lambda s: O.rhs(s, mesh, g2), dt, 2)
        return O.kinetic_energy(qn, mesh)

    qq = q0.clone().requires_grad_(True)
    mu = torch.tensor(gas.mu, dtype=torch.float64, requires_grad=True)
    ke = ke_after(qq, mu)
    gq, gmu = torch.autograd.grad(ke, (qq, mu))
    g = torch.Generator().manual_seed(7)
    u = torch.randn(q0.shape, generator=g, dtype=torch.float64) * q0.abs().amax(dim=(0, 2, 3, 4), keepdim=True)
    h = 1e-6
    fd = (ke_after(q0 + h * u, gas.mu) - ke_after(q0 - h * u, gas.mu)) / (2 * h)
    assert abs(float(fd) - float((gq * u).sum())) < 1e-6 * abs(float(fd))
    hm = 1e-6 * gas.mu
    fdm = (ke_after(q0, gas.mu + hm) - ke_after(q0, gas.mu - hm)) / (2 * hm)
    assert abs(float(fdm) - float(gmu)) < 1e-5 * abs(float(fdm))
