"""Roe-type entropy-stable matrix dissipation (ESDC_DISS_MATRIX) and the interior penalty (ip_coef)
against the oracle's dissipation="matrix" and ip_coef: residual parity under the per-variable
rounding bound used for the ES-C path, with all three volume fluxes, viscous and inviscid; entropy
production between the entropy-conservative and the local Lax-Friedrichs interface terms;
unsupported combinations rejected."""
import pytest
import torch

from oracle import esdc_oracle as O
from tests.gpu_common import assert_parity, make_pair

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
        solver.rhs_vjp(qg, torch.ones_like(qg))
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    s_ip = Solver(2, 2, 2, 2, solver.coords, Re=100.0, ip_coef=1.0)
    with pytest.raises(nat.EsdcError) as ei:
        s_ip.rhs_vjp(qg, torch.ones_like(qg))
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, solver.coords, Re=100.0, precision="fp32", ip_coef=1.0)
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, solver.coords, Re=100.0, ip_coef=-1.0)
    assert ei.value.code == nat.ESDC_ERR_ARG
