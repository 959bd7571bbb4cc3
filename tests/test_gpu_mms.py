"""Bounded boxes with Dirichlet exterior data and a source term (the manufactured-solution setting of
Sec. 5.1) on the GPU: residual parity with the oracle on warped bounded boxes, with all interface
options; the source array is added as given; and the GPU's own manufactured source (esdc_mms_fields)
makes the exact solution's residual vanish at the operator's truncation order; the adjoint on
bounded boxes against the oracle's autograd."""
import math

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I
from tests.gpu_common import assert_parity, normwise_errors

pytestmark = pytest.mark.gpu


def _pair(p, k, warp, Re, **kw):
    from paper_1911_10966_gb300.solver import Solver, lgl
    xi, _ = lgl(p)
    xg = I.box_coords(xi, k, k, k, [0.0] * 3, [1.0] * 3, warp=warp, seed=3)
    solver = Solver(p, k, k, k, xg, Ma=I.MMS_MA, Re=Re, bounded=(True, True, True), **kw)
    s = O.sbp_operator(p)
    xo = I.box_coords(s.xi.numpy(), k, k, k, [0.0] * 3, [1.0] * 3, warp=warp, seed=3)
    mesh = O.make_mesh(p, xo, k, k, k, bounded=(True, True, True))
    gas = O.Gas.from_mach(I.MMS_MA, Re)
    return solver, xg, mesh, xo, gas


@pytest.mark.parametrize("p,k,Re,kw", [(2, 3, 1.0e3, {}), (3, 2, 0.0, {"dissipation": False}),
                                       (4, 2, 4.0e2, {"dissipation": "matrix", "ip_coef": 2.0}),
                                       (3, 2, 1.0e3, {"volume_flux": "kg"}), (2, 2, 1.0e3, {"volume_flux": "dc"})])
def test_bounded_box_parity(p, k, Re, kw):
    """State: the manufactured field with seeded noise; exterior data: the unperturbed field (so the
    boundary terms are active); source: a seeded array, added as given on both sides."""
    solver, xg, mesh, xo, gas = _pair(p, k, 0.1, Re, **kw)
    qg_np = I.perturb(I.manufactured(xg), seed=4, rel=1e-2)
    qo = torch.tensor(I.perturb(I.manufactured(xo), seed=4, rel=1e-2))
    src = I.random_direction(qg_np.shape, seed=5, scale=1.0)
    qg = solver.to_device(qg_np)
    ext = solver.to_device(I.manufactured(xg))
    sg = solver.to_device(src)
    solver.set_exterior(ext)
    solver.set_source(sg)
    ro = O.rhs(qo, mesh, gas, dissipation=kw.get("dissipation", True), scheme=kw.get("volume_flux", "esc"),
               ip_coef=kw.get("ip_coef", 0.0), q_ext=torch.tensor(I.manufactured(xo)), source=torch.tensor(src))
    assert_parity(solver.rhs(qg), ro, qo, mesh, gas)


def test_gpu_manufactured_solution_residual_converges():
    """The GPU residual with the library's own exact exterior data and manufactured source: the L2(PJ)
    norm of R(q_exact) + S relative to S drops at rate >= p - 0.3 (p = 3, k = 4 -> 8)."""
    from paper_1911_10966_gb300.solver import mms_fields
    errs = []
    for k in (4, 8):
        solver, xg, mesh, xo, gas = _pair(3, k, 0.0, I.MMS_RE)
        q, s = mms_fields(xg, I.manufactured_table(), gamma=1.4, Ma=I.MMS_MA, Re=I.MMS_RE, Pr=0.72, L=1.0)
        qd = solver.to_device(q)
        solver.set_exterior(qd)
        sd = solver.to_device(s)
        solver.set_source(sd)
        r = solver.rhs(qd).cpu().numpy()
        J, _ = solver.geometry()
        from paper_1911_10966_gb300.solver import lgl
        _, w = lgl(3)
        PJ = (w[:, None, None] * w[None, :, None] * w[None, None, :])[None] * J
        errs.append(math.sqrt((PJ[:, None] * r ** 2).sum() / (PJ[:, None] * s ** 2).sum()))
    rate = math.log2(errs[0] / errs[1])
    print("GPU MMS truncation", errs, rate)
    assert rate >= 2.7


def test_bounded_box_requirements():
    from paper_1911_10966_gb300 import _native as nat
    from paper_1911_10966_gb300.solver import Solver
    solver, xg, mesh, xo, gas = _pair(2, 2, 0.0, 100.0)
    q = solver.to_device(I.manufactured(xg))
    with pytest.raises(nat.EsdcError) as ei:
        solver.rhs(q)
    assert ei.value.code == nat.ESDC_ERR_ARG
    s32 = Solver(2, 2, 2, 2, xg, Ma=I.MMS_MA, Re=100.0, bounded=(True, False, False), precision="fp32")
    with pytest.raises(nat.EsdcError) as ei:
        s32.rhs(q)
    assert ei.value.code == nat.ESDC_ERR_ARG
    # the adjoint of a bounded box needs the exterior state as well
    with pytest.raises(nat.EsdcError) as ei:
        solver.rhs_vjp(q, torch.ones_like(q))
    assert ei.value.code == nat.ESDC_ERR_ARG
    solver.set_exterior(q)
    assert torch.isfinite(solver.rhs_vjp(q, torch.ones_like(q))).all()


@pytest.mark.parametrize("p,k,Re,kw", [(2, 3, 1.0e3, {}), (3, 2, 0.0, {"dissipation": False}),
                                       (3, 2, 4.0e2, {"volume_flux": "kg"}), (2, 2, 1.0e3, {"volume_flux": "dc"}),
                                       (3, 2, 1.0e3, {"metrics": "optimized"}),
                                       (3, 2, 4.0e2, {"dissipation": "matrix", "ip_coef": 2.0})])
def test_bounded_box_vjp_matches_oracle_autograd(p, k, Re, kw):
    """The adjoint on a warped bounded box (exterior data constant in q, source constant in q)
    against the oracle's autograd VJP of the same residual, and lambda . dR/dmu against the oracle's
    derivative in mu."""
    solver, xg, mesh, xo, gas = _pair(p, k, 0.1, Re, **kw)
    if kw.get("metrics") == "optimized":
        mesh = O.make_mesh(p, xo, k, k, k, bounded=(True, True, True), metrics="optimized")
    qg = solver.to_device(I.perturb(I.manufactured(xg), seed=4, rel=1e-2))
    qo = torch.tensor(I.perturb(I.manufactured(xo), seed=4, rel=1e-2))
    solver.set_exterior(solver.to_device(I.manufactured(xg)))
    src = I.random_direction(tuple(qo.shape), seed=5, scale=1.0)
    solver.set_source(solver.to_device(src))
    lam = torch.randn(qo.shape, generator=torch.Generator().manual_seed(12), dtype=torch.float64)
    qq = qo.clone().requires_grad_(True)
    viscous = Re > 0.0
    mo = torch.tensor(gas.mu, dtype=torch.float64, requires_grad=True)
    g2 = O.Gas(gas.gamma, gas.R, mo, gas.Pr) if viscous else gas
    r = O.rhs(qq, mesh, g2, dissipation=kw.get("dissipation", True), scheme=kw.get("volume_flux", "esc"),
              ip_coef=kw.get("ip_coef", 0.0), q_ext=torch.tensor(I.manufactured(xo)), source=torch.tensor(src))
    grads = torch.autograd.grad(r, (qq, mo) if viscous else (qq,), lam)
    gg, gmu = solver.rhs_vjp(qg, lam.cuda(), want_mu=True)
    e = normwise_errors(gg, grads[0])
    print("bounded vjp vs oracle autograd", ["%.1e" % x for x in e])
    assert max(e) <= 1e-10, e
    if viscous:
        assert abs(gmu - float(grads[1])) <= 1e-10 * abs(float(grads[1])), (gmu, float(grads[1]))


def test_bounded_box_trajectory_gradient_matches_oracle_autograd():
    """Two DP5 steps on a warped bounded p = 3 box with Dirichlet exterior data and a source: the GPU
    adjoint gradient of the final kinetic energy w.r.t. q_0 and mu equals the oracle's autograd
    gradient."""
    from paper_1911_10966_gb300.autograd import KineticEnergy, Trajectory
    solver, xg, mesh, xo, gas = _pair(3, 2, 0.1, 1.0e3)
    qg = solver.to_device(I.perturb(I.manufactured(xg), seed=6, rel=1e-2))
    qo = torch.tensor(I.perturb(I.manufactured(xo), seed=6, rel=1e-2))
    solver.set_exterior(solver.to_device(I.manufactured(xg)))
    src = I.random_direction(tuple(qo.shape), seed=7, scale=1.0)
    solver.set_source(solver.to_device(src))
    dt = 0.5 * solver.dt_cfl(qg, 0.5)
    q0 = qg.clone().requires_grad_(True)
    mu = torch.tensor(solver.mu, dtype=torch.float64, requires_grad=True)
    KineticEnergy.apply(Trajectory.apply(q0, mu, solver, dt, 2), solver).backward()
    qq = qo.clone().requires_grad_(True)
    mo = torch.tensor(gas.mu, dtype=torch.float64, requires_grad=True)
    g2 = O.Gas(gas.gamma, gas.R, mo, gas.Pr)
    qe, so = torch.tensor(I.manufactured(xo)), torch.tensor(src)
    ke = O.kinetic_energy(O.rk_step(qq, lambda s: O.rhs(s, mesh, g2, q_ext=qe, source=so), dt, 2), mesh)
    gqo, gmo = torch.autograd.grad(ke, (qq, mo))
    e = normwise_errors(q0.grad, gqo)
    print("bounded trajectory gradient vs oracle", ["%.1e" % x for x in e], float(mu.grad), float(gmo))
    assert max(e) <= 1e-9, e
    assert abs(float(mu.grad) - float(gmo)) <= 1e-9 * abs(float(gmo))
