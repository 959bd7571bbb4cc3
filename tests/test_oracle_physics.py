"""Pins of the oracle's gas physics: fluxes, entropy variables, log mean, viscous flux (Sec. 4)."""
import math

import mpmath
import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O

GAS = O.Gas.from_mach(0.1, 1600.0)


def _random_states(n, seed, jump=0.2):
    g = torch.Generator().manual_seed(seed)
    rho = 1.0 + jump * (torch.rand(n, generator=g, dtype=torch.float64) - 0.5)
    u = [torch.randn(n, generator=g, dtype=torch.float64) for _ in range(3)]
    T = 1.0 + jump * (torch.rand(n, generator=g, dtype=torch.float64) - 0.5)
    p = rho * GAS.R * T
    q = torch.stack([rho, rho * u[0], rho * u[1], rho * u[2],
                     p / (GAS.gamma - 1) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)], dim=1)
    return q


def _n(nv, seed):
    g = torch.Generator().manual_seed(seed)
    return [torch.randn(nv, generator=g, dtype=torch.float64) for _ in range(3)]


def test_ec_flux_consistency():
    """f_EC(u, u) = f(u) (the two-point flux is consistent with eq. ns_iflux)."""
    q = _random_states(2000, 1)
    n = _n(2000, 2)
    a = O.ec_flux_n(q, q, n, GAS)
    b = O.euler_flux_n(q, n, GAS)
    assert ((a - b).abs() / (b.abs() + 1.0)).max() < 1e-14


def test_ec_flux_symmetry():
    q1, q2 = _random_states(2000, 3), _random_states(2000, 4)
    n = _n(2000, 5)
    a, b = O.ec_flux_n(q1, q2, n, GAS), O.ec_flux_n(q2, q1, n, GAS)
    assert ((a - b).abs() / (a.abs() + 1.0)).max() < 1e-14


@pytest.mark.parametrize("jump", [0.5, 1e-3, 1e-7])
def test_tadmor_entropy_conservation_condition(jump):
    """(w_i - w_j) . f_EC(q_i, q_j) = psi_i - psi_j with psi = rho u.n: the two-point flux is entropy
    conservative for S = -rho s/(gamma-1)."""
    q1, q2 = _random_states(2000, 6, jump), _random_states(2000, 7, jump)
    n = _n(2000, 8)
    w1, w2 = O.entropy_variables(q1, GAS), O.entropy_variables(q2, GAS)
    f = O.ec_flux_n(q1, q2, n, GAS)
    lhs = ((w1 - w2) * f).sum(dim=1)
    psi = lambda q: q[:, 1] * n[0] + q[:, 2] * n[1] + q[:, 3] * n[2]
    rhs = psi(q1) - psi(q2)
    scale = ((w1 - w2).abs() * f.abs()).sum(dim=1) + 1e-300
    assert ((lhs - rhs).abs() / scale).max() < 1e-12


def test_entropy_variables_are_gradient_of_entropy():
    """w = dS/dq checked by central differences of S = -rho s/(gamma-1) (not by its own formula)."""
    q = _random_states(50, 9)
    w = O.entropy_variables(q, GAS)
    for v in range(5):
        h = 1e-6 * q[:, v].abs().clamp(min=1.0)
        qp, qm = q.clone(), q.clone()
        qp[:, v] += h
        qm[:, v] -= h
        fd = (O.entropy_function(qp, GAS) - O.entropy_function(qm, GAS)) / (2 * h)
        assert ((fd - w[:, v]).abs() / (w[:, v].abs() + 1.0)).max() < 1e-6


def test_logmean_against_high_precision():
    mpmath.mp.dps = 50
    rng = np.random.default_rng(11)
    for rel in (1.0, 1e-2, 1e-5, 1e-9, 1e-13, 0.0):
        a = rng.uniform(0.5, 2.0, 200)
        b = a * (1.0 + rel * rng.uniform(-1, 1, 200))
        L = O.logmean(torch.tensor(a), torch.tensor(b)).numpy()
        for ai, bi, Li in zip(a, b, L):
            A, B = mpmath.mpf(ai), mpmath.mpf(bi)
            ex = (A + B) / 2 if A == B else (A - B) / (mpmath.log(A) - mpmath.log(B))
            assert abs(Li - float(ex)) <= 4e-16 * float(ex)


def test_logmean_gradient_against_high_precision():
    """The oracle's log-mean backward (used for the oracle VJP) against mpmath derivatives."""
    mpmath.mp.dps = 50
    rng = np.random.default_rng(12)
    for rel in (1.0, 1e-2, 1e-4, 1e-7, 1e-12, 0.0):
        a = torch.tensor(rng.uniform(0.5, 2.0, 50), requires_grad=True)
        b = (a.detach() * (1.0 + rel * torch.tensor(rng.uniform(-1, 1, 50)))).requires_grad_(True)
        O.logmean(a, b).sum().backward()
        for ai, bi, ga, gb in zip(a.detach().numpy(), b.detach().numpy(), a.grad.numpy(), b.grad.numpy()):
            A, B = mpmath.mpf(ai), mpmath.mpf(bi)
            if A == B:
                ea = eb = mpmath.mpf(0.5)
            else:
                lg = mpmath.log(A) - mpmath.log(B)
                ea = (lg - (A - B) / A) / lg ** 2
                eb = (-lg + (A - B) / B) / lg ** 2
            assert abs(ga - float(ea)) < 1e-12 and abs(gb - float(eb)) < 1e-12


def _probe_C(q, gas):
    """The 15x15 matrix of the linear map g -> F^V(g) at one state (columns by unit vectors)."""
    n = q.shape[0]
    M = torch.zeros(n, 15, 15, dtype=torch.float64)
    for c in range(15):
        g = torch.zeros(n, 3, 5, dtype=torch.float64)
        g[:, c // 5, c % 5] = 1.0
        M[:, :, c] = O.viscous_flux(q, g, gas).reshape(n, 15)
    return M


def test_viscous_flux_symmetric_psd():
    """eq. Fxment: F^V_m = sum_j C_mj dW/dx_j with C_mj = C_jm^T, and the whole block matrix is
    symmetric positive semi-definite (entropy dissipation)."""
    q = _random_states(20, 13)
    M = _probe_C(q, GAS)
    assert (M - M.transpose(1, 2)).abs().max() < 1e-12 * M.abs().max()
    ev = torch.linalg.eigvalsh(M)
    assert ev.min() > -1e-12 * ev.abs().max()
    # mass row and w1 column are zero (no viscous mass flux; F^V does not depend on dw1)
    assert M[:, 0::5, :].abs().max() == 0 and M[:, :, 0::5].abs().max() == 0


def test_viscous_flux_physical_shear_and_heat():
    """With du1/dx2 = s and dT/dx1 = t (via the entropy-variable chain rule), F^V_2 holds the shear
    stress mu s and F^V_1 holds the heat flux kappa t (eq. Fv, eq. tau)."""
    q = _random_states(5, 14)
    rho, u, p, T = O.primitives(q, GAS)
    s, t = 0.7, -0.3
    # w2 = rho u1/p = u1/(R T), w5 = -1/(R T): for fixed T, dw2 = du1/(R T); dT changes w2 and w5
    g = torch.zeros(5, 3, 5, dtype=torch.float64)
    g[:, 1, 1] = s / (GAS.R * T)                        # d/dx2 of w2 with T fixed
    g[:, 0, 4] = t / (GAS.R * T * T)                    # d/dx1 of w5 = -1/(RT)
    g[:, 0, 1] = -u[0] * t / (GAS.R * T * T)            # d/dx1 of w2 = u1/(RT) at fixed u1
    g[:, 0, 2] = -u[1] * t / (GAS.R * T * T)
    g[:, 0, 3] = -u[2] * t / (GAS.R * T * T)
    FV = O.viscous_flux(q, g, GAS)
    mu, kap = GAS.mu, GAS.kappa
    assert torch.allclose(FV[:, 1, 1], torch.full((5,), mu * s, dtype=torch.float64), rtol=1e-12)
    assert torch.allclose(FV[:, 0, 2], torch.full((5,), mu * s, dtype=torch.float64), rtol=1e-12)
    assert torch.allclose(FV[:, 0, 4], mu * s * u[1] + kap * t, rtol=1e-12)
    assert torch.allclose(FV[:, 1, 4], mu * s * u[0], rtol=1e-12)
    assert FV[:, 2].abs().max() < 1e-15


def test_float32_state_rounding_floor_on_taylor_green():
    """The floor under any residual that reads a float32 state: the oracle's exact float64 residual of
    the Taylor-Green state whose perturbation (rho - 1, rho u, rho E - E0) is rounded to float32 once.
    Its mass and energy errors exceed 1e-5 by more than an order of magnitude (the velocity's float32
    rounding times the O(N^2/h) flux-difference scale, against residuals that the divergence-free
    velocity makes small), while the momentum error stays near 1e-5: the 1e-5 per-variable target
    of the float32-mixed form cannot be met for mass and energy on this state by float32 arithmetic of
    any accuracy."""
    from paper_1911_10966_gb300 import inputs as I
    p, k = 4, 8
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, [-math.pi] * 3, [math.pi] * 3, warp=0.1, seed=0)
    mesh = O.make_mesh(p, x, k, k, k)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = torch.tensor(I.taylor_green(x, Ma=0.1))
    ref = torch.tensor([1.0, 0.0, 0.0, 0.0, gas.R / (gas.gamma - 1.0)], dtype=torch.float64).view(1, 5, 1, 1, 1)
    q32 = ref + (q - ref).float().double()
    r = O.rhs(q, mesh, gas)
    r32 = O.rhs(q32, mesh, gas)
    e = [float((r32[:, v] - r[:, v]).abs().max() / r[:, v].abs().max()) for v in range(5)]
    assert e[0] > 1e-4 and e[4] > 1e-4
    assert max(e[1:4]) < 5e-5
