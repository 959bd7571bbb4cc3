"""SF-KG and DC volume-flux variants (ESDC_FLUX_KG, ESDC_FLUX_DC) against the oracle's "kg" and "dc"
schemes: residual parity under the same per-variable rounding bound as the ES-C path, freestream
preservation on the warped mesh, DP5 steps, and the combinations the library does not build
(float32, adjoint) rejected as unsupported."""
import pytest
import torch

from oracle import esdc_oracle as O
from tests.gpu_common import assert_parity, make_pair, normwise_errors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme", ["kg", "dc"])
@pytest.mark.parametrize("p,k,Re,diss", [(1, (3, 3, 2), 1600.0, True), (3, (3, 2, 2), 1600.0, True),
                                         (3, (2, 2, 2), 0.0, False), (4, (2, 2, 3), 400.0, True),
                                         (7, (2, 2, 2), 1600.0, True)])
def test_variant_residual_parity(scheme, p, k, Re, diss):
    solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.1, seed=3, Re=Re, dissipation=diss, noise=1e-2,
                                          volume_flux=scheme)
    assert_parity(solver.rhs(qg), O.rhs(qo, mesh, gas, dissipation=diss, scheme=scheme), qo, mesh, gas)


@pytest.mark.parametrize("scheme", ["kg", "dc"])
def test_variant_freestream_and_dp5_steps(scheme):
    solver, qg, mesh, gas, qo = make_pair(3, (3, 3, 3), warp=0.1, seed=0, state="freestream", volume_flux=scheme)
    r = solver.rhs(qg)
    assert float(r.abs().max()) <= 1e-12 * (1.0 / (1.4 * 0.01))
    solver, qg, mesh, gas, qo = make_pair(2, (3, 3, 3), warp=0.1, seed=1, Re=800.0, volume_flux=scheme)
    dt = solver.dt_cfl(qg, 0.5)
    q0 = qg.clone()
    solver.rk_step(qg, dt, 5)
    qn = O.rk_step(qo, lambda s: O.rhs(s, mesh, gas, scheme=scheme), dt, 5)
    # the increment is dt sum b k over 30 residuals: bounded as for the ES-C path
    e = normwise_errors(qg - q0, qn - qo)
    assert max(e) <= 1e-10, e


def test_variant_unsupported_combinations():
    from paper_1911_10966_gb300 import _native as nat
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(2, (2, 2, 2), Re=100.0, volume_flux="dc")
    with pytest.raises(nat.EsdcError) as ei:
        Solver(2, 2, 2, 2, solver.coords, Re=100.0, precision="fp32", volume_flux="dc")
    assert ei.value.code == nat.ESDC_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        Solver(2, 2, 2, 2, solver.coords, volume_flux="roe")
