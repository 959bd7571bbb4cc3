"""GPU FP64 path vs the CPU oracle, element by element, through the C ABI (libesdc.so).

Tolerance, per variable v: ||R_gpu - R_ora||_inf <= max(1e-12 ||R_ora||_inf, 8 eps T_v), with T_v the
magnitude of the summed flux-difference terms (tests/gpu_common.term_scale).  For generic states
the first bound (the 1e-12 FP64 target) is the active one; for smooth low-Mach states the oracle's
own float64 rounding (about eps T_v, measured by evaluating the volume term in two algebraically
equal orders) is larger than 1e-12 ||R_v|| and the second bound applies.

Workloads: the 4^3 p=3 Taylor-Green case, every degree p = 1..7 on small warped
meshes with strongly perturbed states (both log-mean branches), ragged element counts, and the
16^3 p=4 warped mesh sampled element by element.
"""
import math

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from tests.gpu_common import assert_parity, make_pair, normwise_errors

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.mark.parametrize("Re,diss", [(1600.0, True), (0.0, True), (0.0, False), (1600.0, False)])
def test_rhs_parity_tgv_4cubed_p3(Re, diss):
    solver, qg, mesh, gas, qo = make_pair(3, (4, 4, 4), Re=Re, dissipation=diss)
    rg = solver.rhs(qg)
    ro = O.rhs(qo, mesh, gas, dissipation=diss)
    assert_parity(rg, ro, qo, mesh, gas)


@pytest.mark.parametrize("p", range(1, 8))
def test_rhs_parity_every_degree_warped(p):
    """Warped 3x2x2 mesh (ragged element count for the packed small-p blocks), 5% noise so that
    the log-mean series and logarithm branches both occur; viscous with dissipation."""
    solver, qg, mesh, gas, qo = make_pair(p, (3, 2, 2), warp=0.1, seed=2, Re=100.0, noise=0.05)
    assert_parity(solver.rhs(qg), O.rhs(qo, mesh, gas), qo, mesh, gas)


@pytest.mark.parametrize("k", [(1, 1, 1), (5, 1, 3), (7, 3, 2)])
def test_rhs_parity_ragged_and_degenerate_boxes(k):
    """One element periodic onto itself, and element counts that leave partial CTAs (p = 1, 2)."""
    for p in (1, 2):
        solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.05, seed=3, Re=400.0, noise=0.02)
        assert_parity(solver.rhs(qg), O.rhs(qo, mesh, gas), qo, mesh, gas)


def test_rhs_parity_16cubed_p4_warped_sampled():
    """The 16^3, p = 4 warped Taylor-Green mesh (512k nodes) at full size; the oracle evaluates a
    seeded sample of 48 elements (with their neighbour closure) one by one."""
    solver, qg, mesh, gas, qo = make_pair(4, (16, 16, 16), warp=0.1, seed=0, Re=1600.0)
    rg = solver.rhs(qg)
    E = torch.tensor(np.random.default_rng(5).choice(16 ** 3, 48, replace=False))
    ro = O.rhs(qo, mesh, gas, elems=E)
    assert_parity(rg[E.cuda()], ro, qo, mesh, gas, elems=E)


def test_freestream_preserved_on_warped_mesh():
    """Uniform flow on the 16^3 p=4 warped mesh: |dq/dt| at round-off of the flux scale."""
    solver, qg, mesh, gas, qo = make_pair(4, (16, 16, 16), warp=0.1, seed=0, Re=1600.0, state="freestream")
    r = solver.rhs(qg)
    J, Ja = solver.geometry()
    flux_scale = (1.0 / (1.4 * 0.01)) * np.abs(Ja).max() / J.min()
    assert float(r.abs().max()) <= 1e-12 * flux_scale


def test_entropy_conservation_and_budget_parity():
    """Inviscid EC residual on the warped mesh: sum P J w.dq/dt vanishes to round-off on the GPU,
    the four budgets agree with the oracle's, and the GPU reduction is bitwise reproducible."""
    solver, qg, mesh, gas, qo = make_pair(3, (4, 4, 4), warp=0.1, seed=1, Re=0.0, dissipation=False, noise=1e-2)
    rg = solver.rhs(qg)
    b1 = solver.budgets(qg, rg)
    b2 = solver.budgets(qg, rg)
    assert b1 == b2
    ro = O.rhs(qo, mesh, gas, dissipation=False)
    bo = O.budgets(qo, ro, mesh, gas)
    PJ = O.quadrature_weights(mesh)
    scale = float((PJ * (O.entropy_variables(qo, gas) * ro).sum(dim=1)).abs().sum())
    assert abs(b1[2]) <= 1e-13 * scale
    assert abs(b1[0] - bo[0]) <= 1e-13 * abs(bo[0])
    assert abs(b1[1] - bo[1]) <= 1e-13 * abs(bo[1])
    assert abs(b1[3] - bo[3]) <= 1e-12 * (abs(bo[3]) + 1e-300) + 1e-13 * scale


def test_viscous_budget_and_tgv_dissipation_rate():
    """Viscous TGV: dKE/dt per unit volume from the GPU budget matches the oracle's (and -3 mu/4)."""
    solver, qg, mesh, gas, qo = make_pair(4, (4, 4, 4), Re=1600.0)
    b = solver.budgets(qg, solver.rhs(qg))
    bo = O.budgets(qo, O.rhs(qo, mesh, gas), mesh, gas)
    assert abs(b[3] - bo[3]) <= 1e-11 * abs(bo[3])
    rate = b[3] / (2 * math.pi) ** 3
    assert abs(rate + 0.75 / 1600.0) < 0.02 * 0.75 / 1600.0


def test_rk_step_parity_10_steps():
    """Ten fixed DP5 steps of the 4^3 p=3 Taylor-Green case, viscous, GPU vs oracle."""
    solver, qg, mesh, gas, qo = make_pair(3, (4, 4, 4), Re=1600.0)
    dt = 2.0e-3
    q0 = qg.clone()
    solver.rk_step(qg, dt, 10)
    qn = O.rk_step(qo, lambda s: O.rhs(s, mesh, gas), dt, 10)
    e = normwise_errors(qg - q0, qn - qo)
    print("rk increment normwise", e)
    # the increment is dt * sum b k over 60 residuals: bounded by the residual parity bound times 10
    assert max(e) <= 1e-10, e


def test_dt_cfl_matches_oracle():
    solver, qg, mesh, gas, qo = make_pair(4, (3, 3, 3), warp=0.1, Re=1600.0)
    assert abs(solver.dt_cfl(qg, 0.5) - O.cfl_dt(qo, mesh, gas, 0.5)) <= 1e-13 * O.cfl_dt(qo, mesh, gas, 0.5)


def test_rhs_host_matches_device():
    solver, qg, mesh, gas, qo = make_pair(3, (3, 3, 3), warp=0.1, Re=1600.0)
    rd = solver.rhs(qg).cpu()
    rh = solver.rhs_host(qg.cpu().pin_memory())
    assert torch.equal(rd, rh)


def test_nonphysical_state_reported_without_fault():
    """A NaN and a negative density are reported by the reductions as ESDC_ERR_STATE; the context
    stays usable afterwards."""
    from paper_1911_10966_gb300 import _native as nat
    solver, qg, mesh, gas, qo = make_pair(2, (2, 2, 2), Re=0.0)
    bad = qg.clone()
    bad[0, 0, 0, 0, 0] = float("nan")
    with pytest.raises(nat.EsdcError) as ei:
        solver.budgets(bad)
    assert ei.value.code == nat.ESDC_ERR_STATE
    bad = qg.clone()
    bad[1, 0, 1, 1, 1] = -1.0
    with pytest.raises(nat.EsdcError) as ei:
        solver.dt_cfl(bad)
    assert ei.value.code == nat.ESDC_ERR_STATE
    assert solver.budgets(qg)[1] > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_budgets_async_equals_budgets(precision):
    """esdc_budgets_async writes the same bits as esdc_budgets into device memory (same kernel and
    summation order), with and without dq/dt; a non-physical node is counted in out[4]."""
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(3, (3, 2, 2), warp=0.1, seed=5, Re=800.0, noise=1e-2)
    if precision == "fp32":
        solver = Solver(3, 3, 2, 2, solver.coords, Re=800.0, precision="fp32")
    r = solver.rhs(qg)
    hist = torch.full((3, 5), float("nan"), dtype=torch.float64, device=qg.device)
    solver.budgets_async(qg, hist[0], r)
    solver.budgets_async(qg, hist[1])
    bad = qg.clone()
    bad[1, 0, 1, 1, 1] = -1.0
    bad[2, 3, 0, 0, 0] = float("inf")
    solver.budgets_async(bad, hist[2])
    h = hist.cpu()
    assert tuple(h[0, :4].tolist()) == solver.budgets(qg, r) and h[0, 4] == 0
    assert tuple(h[1, :4].tolist()) == solver.budgets(qg) and h[1, 4] == 0 and h[1, 2] == 0 and h[1, 3] == 0
    assert h[2, 4] == 2


def test_bad_arguments_rejected():
    from paper_1911_10966_gb300 import _native as nat
    solver, qg, mesh, gas, qo = make_pair(2, (2, 2, 2), Re=0.0)
    L = nat.lib()
    assert L.esdc_rhs(solver._ctx, qg.data_ptr(), qg.data_ptr(), None) == nat.ESDC_ERR_ARG   # overlap
    with pytest.raises(ValueError):
        solver.rhs(qg.float())
    ws = torch.empty(8, dtype=torch.uint8, device=qg.device)
    assert L.esdc_rk_step(solver._ctx, qg.data_ptr(), 1e-3, 1, ws.data_ptr(), 8, None) == nat.ESDC_ERR_ARG


def test_rhs_parity_48cubed_p7_full_size_sampled():
    """The largest workload (Taylor-Green 48^3, p = 7: 56.6 M nodes, 2.3 GB of state) at full size:
    float64 residual on 24 seeded elements against the oracle."""
    E = torch.tensor(np.random.default_rng(7).choice(48 ** 3, 24, replace=False))
    solver, qg, mesh, gas, qo = make_pair(7, (48, 48, 48), Re=1600.0, oracle_elems=E)
    rg = solver.rhs(qg)
    ro = O.rhs(qo, mesh, gas, elems=mesh.rows)
    assert_parity(rg[E.cuda()], ro, qo, mesh, gas, elems=mesh.rows)
