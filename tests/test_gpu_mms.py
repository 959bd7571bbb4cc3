"""Bounded boxes with Dirichlet exterior data and a source term (the manufactured-solution setting of
Sec. 5.1) on the GPU: residual parity with the oracle on warped bounded boxes, with all interface
options; the source array is added as given; and the GPU's own manufactured source (esdc_mms_fields)
makes the exact solution's residual vanish at the operator's truncation order."""
import math

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I
from tests.gpu_common import assert_parity

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
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, xg, Ma=I.MMS_MA, Re=100.0, bounded=(True, False, False), precision="fp32")
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    solver.set_exterior(q)
    with pytest.raises(nat.EsdcError) as ei:
        solver.rhs_vjp(q, torch.ones_like(q))
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
