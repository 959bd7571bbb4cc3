"""Hand-written adjoint (esdc_rhs_vjp, esdc_rk_adjoint) against the oracle's autograd VJP and against
central finite differences of the GPU forward path.

Targets: agreement with central differences (h = 1e-6, float64) to 1e-6 relative (Richardson
extrapolated where the plain difference is itself limited, see each test); with the oracle's VJP
per variable to 1e-10 normwise (measured 1e-15 to 2e-13), and with the oracle's trajectory
gradient to 1e-9.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I
from tests.gpu_common import make_pair, normwise_errors

pytestmark = pytest.mark.gpu


def _oracle_vjp(qo, mesh, gas, lam, dissipation=True):
    qq = qo.clone().requires_grad_(True)
    r = O.rhs(qq, mesh, gas, dissipation=dissipation)
    (g,) = torch.autograd.grad(r, qq, lam)
    return g


def _dirs(q, seed):
    g = torch.Generator().manual_seed(seed)
    scale = q.abs().amax(dim=(0, 2, 3, 4), keepdim=True)
    return torch.randn(q.shape, generator=g, dtype=torch.float64) * scale


@pytest.mark.parametrize("p,diss,Re", [(1, True, 300.0), (2, True, 200.0), (3, True, 1600.0), (3, False, 0.0),
                                       (4, True, 100.0), (5, True, 400.0), (6, True, 800.0), (7, True, 1600.0)])
def test_vjp_matches_oracle_autograd(p, diss, Re):
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=3, Re=Re, dissipation=diss, noise=2e-2)
    lam = torch.randn(qo.shape, generator=torch.Generator().manual_seed(11), dtype=torch.float64)
    go = _oracle_vjp(qo, mesh, gas, lam, diss)
    gg = solver.rhs_vjp(qg, lam.cuda())
    e = normwise_errors(gg, go)
    print("vjp vs oracle autograd", ["%.1e" % x for x in e])
    assert max(e) <= 1e-10, e


def _central(f, h):
    """Central difference at h and its Richardson extrapolation from h and 2h (O(h^4))."""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
    return d1, (4 * d1 - d2) / 3


@pytest.mark.parametrize("diss", [False, True])
def test_vjp_dot_product_with_central_differences(diss):
    """<v, (R(q+hu) - R(q-hu))/2h> (GPU forward) = <(dR/dq)^T v, u> (GPU adjoint).
    Without interface dissipation the residual is smooth and the Richardson value from h = 1e-4 and
    2e-4 (truncation O(h^4), rounding ~1e-8) must agree to 1e-6; the plain difference at h = 1e-6
    is limited by the residual's own rounding (eps times the flux-term scale over h, ~1e-6).  With
    the dissipation on, |u.n| and max() add kinks within O(h) of the state, so only the h = 1e-6
    difference is checked (to 1e-5); its exact agreement is covered by the oracle comparison."""
    solver, qg, mesh, gas, qo = make_pair(4, (4, 4, 4), warp=0.1, seed=1, Re=1000.0, Ma=0.5, state="vortex",
                                          box=([-5.0] * 3, [5.0] * 3), dissipation=diss)
    u = _dirs(qo, 1234).cuda()
    v = torch.randn(qo.shape, generator=torch.Generator().manual_seed(7), dtype=torch.float64).cuda()
    fd = lambda h: float((v * solver.rhs(qg + h * u)).sum())
    fd6, _ = _central(fd, 1e-6)
    _, fdr = _central(fd, 1e-4)
    b = float((solver.rhs_vjp(qg, v) * u).sum())
    print("dot product (dissipation %s): adjoint %.12e fd(1e-6) rel %.2e richardson(1e-4) rel %.2e" % (
        diss, b, abs(fd6 - b) / abs(b), abs(fdr - b) / abs(b)))
    assert abs(fd6 - b) <= 1e-5 * abs(b)
    if not diss:
        assert abs(fdr - b) <= 1e-6 * abs(b)


def test_vjp_mu_is_lambda_dot_viscous_residual():
    """R is linear in mu: lambda . dR/dmu = lambda . (R_mu - R_0)/mu, with R_0 the inviscid residual."""
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(3, (3, 3, 3), warp=0.1, seed=4, Re=500.0, noise=1e-2)
    inv = Solver(3, 3, 3, 3, solver.coords, Re=0.0)
    lam = torch.randn(qo.shape, generator=torch.Generator().manual_seed(5), dtype=torch.float64).cuda()
    _, gmu = solver.rhs_vjp(qg, lam, want_mu=True)
    ref = float((lam * (solver.rhs(qg) - inv.rhs(qg))).sum()) / solver.mu
    assert abs(gmu - ref) <= 1e-10 * abs(ref)


def _ke_after(solver, q0, dt, nsteps):
    q = q0.clone()
    solver.rk_step(q, dt, nsteps)
    return solver.budgets(q)[1]


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "vortex_8cubed_p4_50steps_oracle_grad.json")


def test_trajectory_gradient_vortex_8cubed_p4_50_steps():
    """Isentropic vortex (strength 5, axis (1,1,1), drift perpendicular, Ma 0.5) on the 8^3 warped
    p=4 box [-5,5]^3, mu from Re = 1000, 50 DP5 steps at CFL 0.5: d KE(q_50)/d q_0 along seeded
    directions and d KE/d mu from the adjoint vs central differences (h = 1e-6) and vs the oracle's
    gradient through the same 50 steps (tests/golden, written by make_vortex_adjoint_golden.py)."""
    from paper_1911_10966_gb300.solver import Solver
    from paper_1911_10966_gb300.autograd import KineticEnergy, Trajectory
    gold = json.load(open(GOLDEN))
    solver, qg, mesh, gas, qo = make_pair(4, (8, 8, 8), warp=0.1, seed=1, Re=1000.0, Ma=0.5, state="vortex",
                                          box=([-5.0] * 3, [5.0] * 3))
    dt = gold["dt"]
    assert abs(solver.dt_cfl(qg, 0.5) - dt) <= 1e-13 * dt
    nsteps = 50
    q0 = qg.clone().requires_grad_(True)
    mu = torch.tensor(solver.mu, dtype=torch.float64, requires_grad=True)
    qN = Trajectory.apply(q0, mu, solver, dt, nsteps)
    ke = KineticEnergy.apply(qN, solver)
    ke.backward()
    gq, gmu = q0.grad, float(mu.grad)
    h = 1e-6
    for seed in (1234, 99):
        u = _dirs(qo, seed).cuda()
        fd = (_ke_after(solver, qg + h * u, dt, nsteps) - _ke_after(solver, qg - h * u, dt, nsteps)) / (2 * h)
        ad = float((gq * u).sum())
        og = gold["directional"][str(seed)]
        print("d KE/dq0 . u: fd %.12e adjoint %.12e oracle %.12e rel %.2e / %.2e" % (
            fd, ad, og, abs(fd - ad) / abs(fd), abs(og - ad) / abs(og)))
        assert abs(fd - ad) <= 1e-6 * abs(fd)
        assert abs(og - ad) <= 1e-9 * abs(og)
    # mu: KE(q_50) changes by ~1e-7 for a 1e-6 relative step, so the h = 1e-6 difference is
    # rounding-limited (~1e-6); the Richardson value at h = 1e-4 mu is the 1e-6 check
    ke_mu = lambda hh: _ke_after(Solver(4, 8, 8, 8, solver.coords, Ma=0.5, Re=1.0 / (solver.mu + hh)), qg, dt, nsteps)
    fd6, _ = _central(ke_mu, 1e-6 * solver.mu)
    _, fdr = _central(ke_mu, 1e-4 * solver.mu)
    print("d KE/d mu: adjoint %.12e fd(1e-6) rel %.2e richardson(1e-4) rel %.2e" % (
        gmu, abs(fd6 - gmu) / abs(gmu), abs(fdr - gmu) / abs(gmu)))
    assert abs(fd6 - gmu) <= 1e-5 * abs(gmu)
    assert abs(fdr - gmu) <= 1e-6 * abs(gmu)
    assert abs(gold["dke_dmu"] - gmu) <= 1e-9 * abs(gmu)


@pytest.mark.parametrize("p,k", [(3, (3, 3, 2)), (2, (3, 3, 3))])
def test_stage_checkpoints_equal_recomputation(p, k):
    """The reverse sweep from stored stage states (esdc_rk_step_stages / esdc_rk_adjoint_stages) and
    the two that recompute them from per-step checkpoints (the state with its residual, four
    recomputed residuals per step; the state alone, five) evaluate the same VJPs at stage states that
    agree bit for bit, so the gradients agree to rounding (<= 1e-13).  The second mesh has an odd node
    count (27 elements of 27 nodes), so the states inside the checkpoint arrays start at 8-byte aligned
    offsets."""
    solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.1, seed=6, Re=300.0, Ma=0.5, state="vortex",
                                          box=([-5.0] * 3, [5.0] * 3))
    assert (solver.n_nodes % 2 == 1) == (p == 2)
    dt = 0.5 * solver.dt_cfl(qg, 0.5)
    out = {}
    for kind in ("stages", "k1", "state"):
        q = qg.clone()
        ck = solver.rk_step_ckpt(q, dt, 4, stages=kind == "stages", k1=kind == "k1")
        lam = solver.ke_gradient(q)
        g, gmu = solver.rk_adjoint(ck, dt, lam)
        out[kind] = (g.clone(), gmu, q.clone())
    ga, ma, qa = out["stages"]
    for kind in ("k1", "state"):
        gb, mb, qb = out[kind]
        assert torch.equal(qa, qb)
        e = normwise_errors(ga, gb.cpu())
        print("stage checkpoints vs recomputation (%s)" % kind, ["%.1e" % x for x in e], ma, mb)
        assert max(e) <= 1e-13, e
        assert abs(ma - mb) <= 1e-13 * abs(mb)
    # the autograd wrapper takes the same paths
    from paper_1911_10966_gb300.autograd import KineticEnergy, Trajectory
    q0 = qg.clone().requires_grad_(True)
    mu = torch.tensor(solver.mu, dtype=torch.float64, requires_grad=True)
    KineticEnergy.apply(Trajectory.apply(q0, mu, solver, dt, 4, False), solver).backward()
    assert max(normwise_errors(ga, q0.grad.cpu())) <= 1e-13
    assert abs(float(mu.grad) - ma) <= 1e-13 * abs(ma)


def test_trajectory_gradient_matches_oracle_autograd():
    """Three DP5 steps on a 2^3 warped p=3 vortex box: the GPU adjoint gradient of the final kinetic
    energy w.r.t. q_0 and mu equals the oracle's autograd gradient."""
    from paper_1911_10966_gb300.autograd import KineticEnergy, Trajectory
    solver, qg, mesh, gas, qo = make_pair(3, (2, 2, 2), warp=0.1, seed=2, Re=200.0, Ma=0.5, state="vortex",
                                          box=([-5.0] * 3, [5.0] * 3))
    dt = 0.5 * solver.dt_cfl(qg, 0.5)
    q0 = qg.clone().requires_grad_(True)
    mu = torch.tensor(solver.mu, dtype=torch.float64, requires_grad=True)
    KineticEnergy.apply(Trajectory.apply(q0, mu, solver, dt, 3), solver).backward()
    qq = qo.clone().requires_grad_(True)
    mo = torch.tensor(gas.mu, dtype=torch.float64, requires_grad=True)
    g2 = O.Gas(gas.gamma, gas.R, mo, gas.Pr)
    ke = O.kinetic_energy(O.rk_step(qq, lambda s: O.rhs(s, mesh, g2), dt, 3), mesh)
    gqo, gmo = torch.autograd.grad(ke, (qq, mo))
    e = normwise_errors(q0.grad, gqo)
    print("trajectory gradient vs oracle", ["%.1e" % x for x in e], float(mu.grad), float(gmo))
    assert max(e) <= 1e-9, e
    assert abs(float(mu.grad) - float(gmo)) <= 1e-9 * abs(float(gmo))


def test_vjp_and_trajectory_gradient_ignore_a_constant_source():
    """A source term is constant in q: the VJP is unchanged bit for bit, and the trajectory gradient
    through DP5 steps with the source (whose stages do depend on it) matches the oracle's autograd."""
    solver, qg, mesh, gas, qo = make_pair(3, (2, 2, 2), warp=0.1, seed=4, Re=400.0, noise=1e-2)
    lam = torch.randn(qo.shape, generator=torch.Generator().manual_seed(13), dtype=torch.float64).cuda()
    g0 = solver.rhs_vjp(qg, lam)
    src = torch.tensor(I.random_direction(tuple(qo.shape), seed=21, scale=1.0), device=qg.device)
    solver.set_source(src)
    g1 = solver.rhs_vjp(qg, lam)
    assert torch.equal(g0, g1)
    dt = 0.5 * solver.dt_cfl(qg, 0.5)
    from paper_1911_10966_gb300.autograd import Trajectory, KineticEnergy
    q0 = qg.clone().requires_grad_(True)
    mu = torch.tensor(solver.mu, dtype=torch.float64, requires_grad=True)
    KineticEnergy.apply(Trajectory.apply(q0, mu, solver, dt, 2), solver).backward()
    so = src.cpu()
    qq = qo.clone().requires_grad_(True)
    qn = O.rk_step(qq, lambda s: O.rhs(s, mesh, gas, source=so), dt, 2)
    ke = O.kinetic_energy(qn, mesh)
    (go,) = torch.autograd.grad(ke, qq)
    e = normwise_errors(q0.grad, go)
    assert max(e) <= 1e-9, e


@pytest.mark.parametrize("vf,p,diss,Re", [("kg", 2, True, 200.0), ("kg", 3, False, 0.0), ("kg", 4, True, 800.0),
                                          ("kg", 7, True, 1600.0), ("dc", 2, True, 200.0), ("dc", 3, True, 400.0),
                                          ("dc", 4, False, 0.0), ("dc", 6, True, 800.0)])
def test_variant_vjp_matches_oracle_autograd(vf, p, diss, Re):
    """The adjoint of the SF-KG (Kennedy-Gruber two-point flux) and DC (nodal Euler fluxes, central
    interface flux) variants against the oracle's autograd VJP, and a two-step trajectory gradient
    against the oracle's."""
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=3, Re=Re, dissipation=diss, noise=2e-2,
                                          volume_flux=vf)
    lam = torch.randn(qo.shape, generator=torch.Generator().manual_seed(14), dtype=torch.float64)
    qq = qo.clone().requires_grad_(True)
    (go,) = torch.autograd.grad(O.rhs(qq, mesh, gas, dissipation=diss, scheme=vf), qq, lam)
    e = normwise_errors(solver.rhs_vjp(qg, lam.cuda()), go)
    assert max(e) <= 1e-10, e
    if p != 3:
        return
    from paper_1911_10966_gb300.autograd import Trajectory, KineticEnergy
    dt = 0.5 * solver.dt_cfl(qg, 0.5)
    q0 = qg.clone().requires_grad_(True)
    mu = torch.tensor(solver.mu, dtype=torch.float64, requires_grad=True)
    KineticEnergy.apply(Trajectory.apply(q0, mu, solver, dt, 2), solver).backward()
    qq = qo.clone().requires_grad_(True)
    ke = O.kinetic_energy(O.rk_step(qq, lambda s: O.rhs(s, mesh, gas, dissipation=diss, scheme=vf), dt, 2), mesh)
    (gt,) = torch.autograd.grad(ke, qq)
    e = normwise_errors(q0.grad, gt)
    assert max(e) <= 1e-9, e


def test_checkpoint_argument_checks():
    """Checkpoints holding the first residual are a float64 feature: a float32-mixed context refuses
    them; a checkpoint tensor of the wrong shape is refused before any launch."""
    from paper_1911_10966_gb300 import _native as nat
    s32, q32, _, _, _ = make_pair(3, (2, 2, 2), Re=400.0, precision="fp32", noise=1e-3)
    with pytest.raises(nat.EsdcError) as ei:
        s32.rk_step_ckpt(q32.clone(), 1e-4, 2, k1=True)
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    solver, qg, _, _, _ = make_pair(3, (2, 2, 2), Re=400.0, noise=1e-3)
    bad = torch.zeros((2, 3) + tuple(qg.shape), dtype=torch.float64, device=qg.device)
    with pytest.raises(ValueError):
        solver.rk_adjoint(bad, 1e-4, torch.ones_like(qg))
