"""The paper's optimized metrics (Sec. 3; ESDC_METRICS_OPTIMIZED) on the GPU against the oracle:
residual parity on warped periodic meshes with every volume flux and interface option, on a sample of
the 16^3 p = 4 warped Taylor-Green mesh, and on bounded boxes with exterior data and a source; a
uniform flow stays steady; unsupported combinations are refused."""
import math

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I
from tests.gpu_common import assert_parity, make_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,k,Re,vf,kw", [(1, (3, 3, 2), 1600.0, "esc", {}), (3, (3, 2, 2), 0.0, "esc", {}),
                                          (4, (2, 2, 3), 400.0, "esc", {"dissipation": "matrix"}),
                                          (7, (2, 2, 2), 1600.0, "esc", {}), (3, (2, 3, 2), 800.0, "kg", {}),
                                          (3, (2, 2, 2), 0.0, "dc", {}), (2, (3, 3, 2), 200.0, "esc", {"ip_coef": 1.0}),
                                          (2, (2, 2, 2), 0.0, "esc", {"dissipation": False})])
def test_optimized_metrics_parity(p, k, Re, vf, kw):
    from paper_1911_10966_gb300.solver import Solver
    diss = kw.get("dissipation", True)
    solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.1, seed=5, Re=Re, dissipation=diss, noise=2e-2,
                                          volume_flux=vf, metrics="optimized")
    if kw.get("ip_coef"):
        solver = Solver(p, *k, solver.coords, Re=Re, dissipation=diss, ip_coef=kw["ip_coef"], metrics="optimized")
    ro = O.rhs(qo, mesh, gas, dissipation=diss, scheme=vf, ip_coef=kw.get("ip_coef", 0.0))
    assert_parity(solver.rhs(qg), ro, qo, mesh, gas)


def test_optimized_metrics_sampled_parity_16cubed_p4():
    """The 16^3 p = 4 warped Taylor-Green mesh (seed 0): 6 sampled elements, including periodic-wrap
    ones, against the oracle on their two-ring submesh."""
    E = torch.tensor([0, 15, 255, 2048, 3839, 4095])
    solver, qg, mesh, gas, qo = make_pair(4, (16, 16, 16), warp=0.1, seed=0, Re=1600.0, oracle_elems=E,
                                          metrics="optimized")
    ro = O.rhs(qo, mesh, gas, elems=mesh.rows)
    assert_parity(solver.rhs(qg)[E.to(qg.device)], ro, qo, mesh, gas, elems=mesh.rows)


@pytest.mark.parametrize("p", [2, 4])
def test_optimized_metrics_freestream(p):
    solver, qg, mesh, gas, qo = make_pair(p, (3, 3, 3), warp=0.1, seed=2, Ma=0.3, Re=200.0, state="freestream",
                                          metrics="optimized")
    r = solver.rhs(qg)
    assert float(r.abs().max()) < 1e-11 * gas.R


def test_optimized_metrics_bounded_box_parity():
    from paper_1911_10966_gb300.solver import Solver, lgl
    p, k, Re = 3, 2, 1.0e3
    xi, _ = lgl(p)
    xg = I.box_coords(xi, k, k, k, [0.0] * 3, [1.0] * 3, warp=0.1, seed=3)
    solver = Solver(p, k, k, k, xg, Ma=I.MMS_MA, Re=Re, bounded=(True, True, True), metrics="optimized")
    s = O.sbp_operator(p)
    xo = I.box_coords(s.xi.numpy(), k, k, k, [0.0] * 3, [1.0] * 3, warp=0.1, seed=3)
    mesh = O.make_mesh(p, xo, k, k, k, bounded=(True, True, True), metrics="optimized")
    gas = O.Gas.from_mach(I.MMS_MA, Re)
    qg = solver.to_device(I.perturb(I.manufactured(xg), seed=4, rel=1e-2))
    qo = torch.tensor(I.perturb(I.manufactured(xo), seed=4, rel=1e-2))
    src = I.random_direction(qo.shape, seed=5, scale=1.0)
    solver.set_exterior(solver.to_device(I.manufactured(xg)))
    solver.set_source(solver.to_device(src))
    ro = O.rhs(qo, mesh, gas, q_ext=torch.tensor(I.manufactured(xo)), source=torch.tensor(src))
    assert_parity(solver.rhs(qg), ro, qo, mesh, gas)


def test_optimized_metrics_unsupported():
    from paper_1911_10966_gb300 import _native as nat
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(2, (2, 2, 2), warp=0.1, Re=100.0, metrics="optimized")
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, solver.coords, Re=100.0, precision="fp32", metrics="optimized", volume_flux="dc")
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        Solver(2, 2, 2, 2, solver.coords, metrics="exact")


@pytest.mark.parametrize("p,diss,Re", [(3, True, 800.0), (2, False, 0.0), (4, True, 200.0)])
def test_optimized_metrics_vjp_matches_oracle_autograd(p, diss, Re):
    """The hand-written adjoint with the surface metrics in its interface terms against the oracle's
    autograd VJP of the optimized-metric residual."""
    from tests.gpu_common import normwise_errors
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=3, Re=Re, dissipation=diss, noise=2e-2,
                                          metrics="optimized")
    lam = torch.randn(qo.shape, generator=torch.Generator().manual_seed(12), dtype=torch.float64)
    qq = qo.clone().requires_grad_(True)
    (go,) = torch.autograd.grad(O.rhs(qq, mesh, gas, dissipation=diss), qq, lam)
    e = normwise_errors(solver.rhs_vjp(qg, lam.cuda()), go)
    assert max(e) <= 1e-10, e


def test_optimized_metrics_dp5_steps():
    """Five fixed DP5 steps, viscous, warped mesh, optimized metrics: the increment against the
    oracle's."""
    from tests.gpu_common import normwise_errors
    solver, qg, mesh, gas, qo = make_pair(3, (3, 2, 2), warp=0.1, seed=6, Re=800.0, metrics="optimized")
    dt = solver.dt_cfl(qg, 0.5)
    q0 = qg.clone()
    solver.rk_step(qg, dt, 5)
    qn = O.rk_step(qo, lambda s: O.rhs(s, mesh, gas), dt, 5)
    e = normwise_errors(qg - q0, qn - qo)
    assert max(e) <= 1e-10, e
