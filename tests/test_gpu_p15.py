"""p = 15 (N = 16, the top degree of the paper's cost comparison, Sec. 5.3): the multi-pass float64
residual against the oracle on warped periodic meshes with the ES-C, SF-KG and DC volume fluxes,
viscous and inviscid, entropy conservation of the EC scheme, a uniform flow kept, a DP5 step and
the budgets; combinations not built at this degree refused.

The parity bound adds geometry_rounding(p) T_v: at p = 15 the two sides' curl-form metrics, each
float64-exact to round-off amplified by |D|^2 (|D| = 60), differ by ~1e-11 relative."""
import math

import pytest
import torch

from oracle import esdc_oracle as O
from tests.gpu_common import assert_parity, geometry_rounding, make_pair, normwise_errors

pytestmark = pytest.mark.gpu

P = 15


@pytest.mark.parametrize("k,Re,vf,diss", [((2, 2, 2), 1600.0, "esc", True), ((2, 1, 2), 0.0, "esc", False),
                                          ((2, 2, 1), 800.0, "kg", True), ((1, 2, 2), 0.0, "dc", True),
                                          ((2, 2, 2), 400.0, "dc", False), ((1, 1, 1), 1600.0, "esc", True)])
def test_p15_residual_parity(k, Re, vf, diss):
    solver, qg, mesh, gas, qo = make_pair(P, k, warp=0.1, seed=4, Re=Re, dissipation=diss, noise=2e-2,
                                          volume_flux=vf)
    ro = O.rhs(qo, mesh, gas, dissipation=diss, scheme=vf)
    assert_parity(solver.rhs(qg), ro, qo, mesh, gas, geo_rel=geometry_rounding(P))


def test_p15_entropy_conservation_and_budgets():
    """Inviscid EC residual: sum P J w.dq/dt vanishes to round-off on the GPU; the four budgets agree
    with the oracle's."""
    solver, qg, mesh, gas, qo = make_pair(P, (2, 2, 2), warp=0.1, seed=1, Re=0.0, dissipation=False, noise=1e-2)
    rg = solver.rhs(qg)
    b = solver.budgets(qg, rg)
    ro = O.rhs(qo, mesh, gas, dissipation=False)
    bo = O.budgets(qo, ro, mesh, gas)
    PJ = O.quadrature_weights(mesh)
    scale = float((PJ * (O.entropy_variables(qo, gas) * ro).sum(dim=1)).abs().sum())
    assert abs(b[2]) <= 1e-12 * scale
    assert abs(b[0] - bo[0]) <= 1e-13 * abs(bo[0])
    assert abs(b[1] - bo[1]) <= 1e-13 * abs(bo[1])
    assert abs(b[3] - bo[3]) <= 1e-12 * scale


def test_p15_freestream():
    """Uniform flow on the warped mesh: |dq/dt| at the round-off of the metric terms (the oracle's own
    value is 2e-12 of the pressure scale R here)."""
    solver, qg, mesh, gas, qo = make_pair(P, (2, 2, 2), warp=0.1, seed=2, Re=1600.0, state="freestream")
    r = solver.rhs(qg)
    assert float(r.abs().max()) <= geometry_rounding(P) * gas.R


def test_p15_dp5_step():
    """Two DP5 steps, viscous, GPU vs oracle: the increment's normwise error stays at the residual's
    parity level."""
    solver, qg, mesh, gas, qo = make_pair(P, (2, 2, 2), warp=0.1, seed=3, Re=1600.0)
    dt = 0.5 * solver.dt_cfl(qg, 0.5)
    q0 = qg.clone()
    solver.rk_step(qg, dt, 2)
    qn = O.rk_step(qo, lambda s: O.rhs(s, mesh, gas), dt, 2)
    e = normwise_errors(qg - q0, qn - qo)
    print("p = 15 increment normwise", e)
    assert max(e) <= 1e-8, e


def test_p15_unsupported_combinations():
    from paper_1911_10966_gb300 import _native as nat
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(P, (1, 1, 1), Re=100.0)
    for kw in (dict(precision="fp32"), dict(dissipation="matrix"), dict(ip_coef=1.0), dict(metrics="optimized"),
               dict(bounded=(True, False, False))):
        with pytest.raises(nat.EsdcError) as ei:
            Solver(P, 1, 1, 1, solver.coords, Re=100.0, **kw)
        assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED, kw
    with pytest.raises(nat.EsdcError) as ei:
        solver.rhs_vjp(qg, torch.ones_like(qg))
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED


def test_p15_adaptive_matches_oracle():
    """Adaptive DP5(4) at p = 15 (one element periodic onto itself): the same accepted and rejected
    steps as the oracle's integrator and the same final state (tolerances of the p <= 7 test)."""
    solver, qg, mesh, gas, qo = make_pair(P, (1, 1, 1), warp=0.1, seed=2, Re=200.0, noise=1e-2)
    dt_cfl = solver.dt_cfl(qg, 0.5)
    st = solver.rk_adaptive(qg, 0.0, 6.0 * dt_cfl, 3.0 * dt_cfl, rtol=1e-6, atol=1e-6, max_steps=200, history=500)
    qo_end, so = O.rk_adaptive(qo, lambda s: O.rhs(s, mesh, gas), 0.0, 6.0 * dt_cfl, 3.0 * dt_cfl, 1e-6, 1e-6,
                               max_steps=200)
    assert st["accepted"] == len(so["accepted"]) and st["rejected"] == so["rejected"]
    for a, b in zip(st["dt_history"], so["accepted"]):
        assert abs(a - b) <= 1e-8 * b
    e = normwise_errors(qg, qo_end)
    assert max(e) <= 1e-9, e


def test_p15_source_term_parity():
    """A seeded source array is added to dq/dt at p = 15 as at p <= 7: parity with the oracle's
    residual with the same source, under the p = 15 bound."""
    from paper_1911_10966_gb300 import inputs as I
    solver, qg, mesh, gas, qo = make_pair(P, (1, 1, 2), warp=0.1, seed=4, Re=800.0, noise=2e-2)
    src = I.random_direction(tuple(qo.shape), seed=6, scale=1.0)
    solver.set_source(solver.to_device(src))
    ro = O.rhs(qo, mesh, gas, source=torch.tensor(src))
    assert_parity(solver.rhs(qg), ro, qo, mesh, gas, geo_rel=geometry_rounding(P))
