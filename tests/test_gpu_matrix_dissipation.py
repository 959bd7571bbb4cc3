"""Roe-type entropy-stable matrix dissipation (ESDC_DISS_MATRIX) and the interior penalty (ip_coef)
against the oracle's dissipation="matrix" and ip_coef: residual parity under the per-variable
rounding bound used for the ES-C path, with all three volume fluxes, viscous and inviscid; entropy
production between the entropy-conservative and the local Lax-Friedrichs interface terms;
unsupported combinations rejected; the adjoint of both terms against the oracle's autograd."""
import pytest
import torch

from oracle import esdc_oracle as O
from tests.gpu_common import assert_parity, make_pair, normwise_errors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,k,Re,vf", [(1, (3, 3, 2), 1600.0, "esc"), (3, (3, 2, 2), 0.0, "esc"),
                                       (4, (2, 2, 3), 400.0, "esc"), (7, (2, 2, 2), 1600.0, "esc"),
                                       (3, (2, 3, 2), 800.0, "kg"), (3, (2, 2, 2), 0.0, "dc")])
def test_matrix_dissipation_parity(p, k, Re, vf):
    solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.1, seed=5, Re=Re, dissipation="matrix", noise=2e-2,
                                          volume_flux=vf)
    ro = O.rhs(qo, mesh, gas, dissipation="matrix", scheme=vf)
    assert_parity(solver.rhs(qg), ro, qo, mesh, gas)


@pytest.mark.parametrize("p,k,Re,diss,ip", [(3, (3, 2, 2), 400.0, True, 1.0), (4, (2, 2, 2), 1600.0, "matrix", 4.0),
                                            (2, (3, 3, 2), 200.0, False, 0.5)])
def test_interior_penalty_parity(p, k, Re, diss, ip):
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.1, seed=8, Re=Re, dissipation=diss, noise=2e-2)
    s_ip = Solver(p, *k, solver.coords, Re=Re, dissipation=diss, ip_coef=ip)
    assert_parity(s_ip.rhs(qg), O.rhs(qo, mesh, gas, dissipation=diss, ip_coef=ip), qo, mesh, gas)


def test_matrix_dissipation_entropy_budget():
    """Inviscid, noisy Taylor-Green state: sum P J w.dq/dt from the GPU budgets is negative and lies
    between the local Lax-Friedrichs value and zero (the entropy-conservative value)."""
    out = {}
    for diss in (False, True, "matrix"):
        solver, qg, mesh, gas, qo = make_pair(3, (3, 3, 3), warp=0.1, seed=6, Re=0.0, Ma=0.3, dissipation=diss,
                                              noise=5e-2)
        out[diss] = solver.budgets(qg, solver.rhs(qg))[2]
    assert out[True] < out["matrix"] < 0.0
    assert abs(out[False]) <= 1e-6 * abs(out["matrix"])


def test_matrix_dissipation_unsupported_combinations():
    from paper_1911_10966_gb300 import _native as nat
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(2, (2, 2, 2), Re=100.0, dissipation="matrix")
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, solver.coords, Re=100.0, precision="fp32", dissipation="matrix")
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, solver.coords, Re=100.0, precision="fp32", ip_coef=1.0)
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, solver.coords, Re=100.0, ip_coef=-1.0)
    assert ei.value.code == nat.ESDC_ERR_ARG


def _oracle_grads(qo, mesh, gas, lam, viscous, **kw):
    """(dR/dq)^T lam and lam . dR/dmu of the oracle's residual by autograd."""
    qq = qo.clone().requires_grad_(True)
    mo = torch.tensor(gas.mu, dtype=torch.float64, requires_grad=True)
    g2 = O.Gas(gas.gamma, gas.R, mo, gas.Pr) if viscous else gas
    grads = torch.autograd.grad(O.rhs(qq, mesh, g2, **kw), (qq, mo) if viscous else (qq,), lam)
    return grads[0], (float(grads[1]) if viscous else None)


@pytest.mark.parametrize("p,k,Re,diss,ip,vf", [(2, (3, 2, 2), 400.0, "matrix", 0.0, "esc"),
                                               (3, (2, 2, 2), 0.0, "matrix", 0.0, "esc"),
                                               (4, (2, 2, 2), 1600.0, "matrix", 0.0, "kg"),
                                               (3, (2, 2, 2), 400.0, "matrix", 0.0, "dc"),
                                               (3, (3, 2, 2), 400.0, True, 1.0, "esc"),
                                               (2, (2, 2, 3), 200.0, False, 0.5, "esc"),
                                               (4, (2, 2, 2), 800.0, "matrix", 4.0, "esc")])
def test_matrix_dissipation_and_interior_penalty_vjp(p, k, Re, diss, ip, vf):
    """The adjoint with the Roe-type matrix dissipation and/or the interior penalty against the
    oracle's autograd VJP; lam . dR/dmu (the penalty is linear in mu) against the oracle's."""
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.1, seed=9, Re=Re, dissipation=diss, noise=2e-2,
                                          volume_flux=vf)
    if ip > 0.0:
        solver = Solver(p, *k, solver.coords, Re=Re, dissipation=diss, ip_coef=ip, volume_flux=vf)
    lam = torch.randn(qo.shape, generator=torch.Generator().manual_seed(15), dtype=torch.float64)
    go, gmo = _oracle_grads(qo, mesh, gas, lam, Re > 0.0, dissipation=diss, scheme=vf, ip_coef=ip)
    gg, gmu = solver.rhs_vjp(qg, lam.cuda(), want_mu=True)
    e = normwise_errors(gg, go)
    print("matrix/IP vjp vs oracle autograd", ["%.1e" % x for x in e], gmu, gmo)
    assert max(e) <= 1e-10, e
    if gmo is not None:
        assert abs(gmu - gmo) <= 1e-10 * abs(gmo), (gmu, gmo)


def test_matrix_dissipation_interior_penalty_trajectory_gradient():
    """Two DP5 steps with matrix dissipation and the interior penalty: the GPU adjoint gradient of the
    final kinetic energy w.r.t. q_0 and mu equals the oracle's autograd gradient."""
    from paper_1911_10966_gb300.autograd import KineticEnergy, Trajectory
    from paper_1911_10966_gb300.solver import Solver
    s0, qg, mesh, gas, qo = make_pair(3, (2, 2, 2), warp=0.1, seed=10, Re=400.0, dissipation="matrix", noise=2e-2)
    solver = Solver(3, 2, 2, 2, s0.coords, Re=400.0, dissipation="matrix", ip_coef=2.0)
    dt = 0.5 * solver.dt_cfl(qg, 0.5)
    q0 = qg.clone().requires_grad_(True)
    mu = torch.tensor(solver.mu, dtype=torch.float64, requires_grad=True)
    KineticEnergy.apply(Trajectory.apply(q0, mu, solver, dt, 2), solver).backward()
    qq = qo.clone().requires_grad_(True)
    mo = torch.tensor(gas.mu, dtype=torch.float64, requires_grad=True)
    g2 = O.Gas(gas.gamma, gas.R, mo, gas.Pr)
    ke = O.kinetic_energy(O.rk_step(qq, lambda s: O.rhs(s, mesh, g2, dissipation="matrix", ip_coef=2.0), dt, 2),
                          mesh)
    gqo, gmo = torch.autograd.grad(ke, (qq, mo))
    e = normwise_errors(q0.grad, gqo)
    print("matrix/IP trajectory gradient vs oracle", ["%.1e" % x for x in e], float(mu.grad), float(gmo))
    assert max(e) <= 1e-9, e
    assert abs(float(mu.grad) - float(gmo)) <= 1e-9 * abs(float(gmo))
