"""Manufactured solution with Dirichlet boundaries (Sec. 5.1, eq. mms): the oracle's boundary SATs and
autograd source are consistent (the residual of the exact solution plus the source vanishes at the
order of the operator's truncation error), a freestream is preserved on a bounded box with its own
state as the exterior data, and the library's host-side analytic source (esdc_mms_fields) equals the
oracle's autograd source."""
import math

import numpy as np
import pytest
import torch

from oracle import esdc_oracle as O
from paper_1911_10966_gb300 import inputs as I

F64 = torch.float64
PRIM = lambda a, b, c: I.manufactured_primitives(a, b, c, sin=torch.sin, cos=torch.cos)


def _mms(p, k, warp=0.0):
    s = O.sbp_operator(p)
    x = I.box_coords(s.xi.numpy(), k, k, k, [0.0] * 3, [1.0] * 3, warp=warp, seed=3)
    mesh = O.make_mesh(p, x, k, k, k, bounded=(True, True, True))
    return mesh, x


@pytest.mark.parametrize("p", [2, 3])
def test_exact_solution_residual_converges(p):
    """L2(PJ) norm of R(q_exact) + S relative to S: rate >= p - 0.3 from k = 4 to 8 (the collocation
    operator's truncation order p; the boundary SATs and the source must be consistent for it)."""
    gas = O.Gas.from_mach(I.MMS_MA, I.MMS_RE)
    errs = []
    for k in (2, 4, 8):
        mesh, x = _mms(p, k)
        q = torch.tensor(I.manufactured(x))
        S = O.manufactured_source(PRIM, x, gas)
        r = O.rhs(q, mesh, gas, q_ext=q, source=S)
        PJ = O.quadrature_weights(mesh).unsqueeze(1)
        errs.append(float(torch.sqrt((PJ * r ** 2).sum() / (PJ * S ** 2).sum())))
    rate = math.log2(errs[1] / errs[2])
    assert rate >= p - 0.3, (errs, rate)


def test_bounded_box_freestream_and_missing_exterior():
    gas = O.Gas.from_mach(0.5, 100.0)
    mesh, x = _mms(3, 3, warp=0.1)
    qf = torch.tensor(I.freestream(x, Ma=0.5))
    r = O.rhs(qf, mesh, gas, q_ext=qf, ip_coef=1.0, dissipation="matrix")
    assert float(r.abs().max()) < 1e-11 * gas.R
    with pytest.raises(ValueError):
        O.rhs(qf, mesh, gas)


def test_library_mms_fields_match_inputs_and_oracle_source():
    """esdc_mms_fields (host C++, hand-derived derivatives) against the inputs module's field and the
    oracle's autograd divergence, on a warped mesh so that no point lies on a symmetry line."""
    from paper_1911_10966_gb300.solver import mms_fields
    gas = O.Gas.from_mach(I.MMS_MA, 1.0e2)           # a low Re so that the viscous part matters
    mesh, x = _mms(3, 2, warp=0.1)
    q, s = mms_fields(x, I.manufactured_table(), gamma=1.4, Ma=I.MMS_MA, Re=1.0e2, Pr=0.72, L=1.0)
    assert np.allclose(q, I.manufactured(x), rtol=1e-14, atol=0.0)
    so = O.manufactured_source(PRIM, x, gas).numpy()
    for v in range(5):
        assert np.abs(s[:, v] - so[:, v]).max() <= 1e-11 * np.abs(so[:, v]).max(), v
