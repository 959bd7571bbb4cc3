"""esdc_init_state: the library's device-side initial states against the input module's host
versions on the same node coordinates (Taylor-Green, isentropic vortex about an axis with drift,
uniform state), and its argument checks."""
import math

import numpy as np
import pytest
import torch

from paper_1911_10966_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.detach().cpu().numpy()
    return max(float(np.abs(a[:, v] - b[:, v]).max() / np.abs(b[:, v]).max()) if np.abs(b[:, v]).max() > 0
               else float(np.abs(a[:, v]).max()) for v in range(5))


def test_taylor_green_and_freestream_match_inputs():
    from paper_1911_10966_gb300.solver import Solver
    s = Solver.box(3, 3, 2, 2, warp=0.1, seed=2, Ma=0.1, Re=1600.0)
    assert _rel(s.init_state("tgv"), I.taylor_green(s.coords, Ma=0.1)) <= 1e-14
    assert _rel(s.init_state("freestream"), I.freestream(s.coords, Ma=0.1)) <= 1e-15
    q = s.init_state("freestream", params=[1.2, -0.1, 0.0, 0.4, 50.0])
    assert _rel(q, I.freestream(s.coords, rho=1.2, u=(-0.1, 0.0, 0.4), p=50.0, Ma=0.1)) <= 1e-15


def test_vortex_matches_inputs():
    from paper_1911_10966_gb300.solver import Solver
    s = Solver.box(4, 3, 3, 3, lo=(-5.0,) * 3, hi=(5.0,) * 3, warp=0.1, seed=1, Ma=0.5, Re=1000.0)
    u_inf = (1 / math.sqrt(2), -1 / math.sqrt(2), 0.0)
    want = I.isentropic_vortex(s.coords, Ma=0.5, u_inf=u_inf)
    got = s.init_state("vortex", params=[5.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, *u_inf])
    assert _rel(got, want) <= 1e-14
    want = I.isentropic_vortex(s.coords, Ma=0.5, beta=3.0, center=(0.5, -1.0, 0.25), axis=(0.0, 0.0, 2.0))
    got = s.init_state("vortex", params=[3.0, 0.5, -1.0, 0.25, 0.0, 0.0, 2.0, 0.0, 0.0, 0.0])
    assert _rel(got, want) <= 1e-14
    assert _rel(s.init_state("vortex"), I.isentropic_vortex(s.coords, Ma=0.5)) <= 1e-14


def test_init_state_argument_errors():
    from paper_1911_10966_gb300 import _native as nat
    from paper_1911_10966_gb300.solver import Solver
    s = Solver.box(2, 2, 2, 2, Ma=0.3)
    q = s.init_state()
    L = nat.lib()
    assert L.esdc_init_state(s._ctx, 7, None, q.data_ptr(), None) == nat.ESDC_ERR_ARG
    assert L.esdc_init_state(s._ctx, 0, None, None, None) == nat.ESDC_ERR_ARG
    zero_axis = np.array([5.0, 0, 0, 0, 0, 0, 0, 0, 0, 0])
    assert L.esdc_init_state(s._ctx, 1, zero_axis.ctypes.data, q.data_ptr(), None) == nat.ESDC_ERR_ARG
    bad = np.array([1.0, 0.0, 0.0, 0.0, -1.0])
    assert L.esdc_init_state(s._ctx, 2, bad.ctypes.data, q.data_ptr(), None) == nat.ESDC_ERR_ARG
    with pytest.raises(ValueError):
        s.init_state("shock")
    with pytest.raises(ValueError):
        s.init_state("vortex", params=[1.0, 2.0])


def test_generated_mesh_residual_parity():
    """esdc_create without node coordinates (the library's box generator): the residual of a device
    Taylor-Green state on the warped generated mesh against the oracle on the input module's mesh
    built with the same splitmix64 phases."""
    from oracle import esdc_oracle as O
    from paper_1911_10966_gb300.solver import Solver
    from tests.gpu_common import assert_parity
    p, k, seed = 3, (3, 2, 2), 11
    lo, hi = (-math.pi,) * 3, (math.pi,) * 3
    s = Solver(p, *k, None, Re=1600.0, lo=lo, hi=hi, warp=0.1, seed=seed)
    xo = I.box_coords(O.sbp_operator(p).xi.numpy(), *k, lo, hi, warp=0.1, phases=I.splitmix64_phases(seed))
    assert np.abs(s.coords - xo).max() <= 1e-15 * np.abs(xo).max()
    mesh = O.make_mesh(p, xo, *k)
    gas = O.Gas.from_mach(0.1, 1600.0)
    q = s.init_state("tgv")
    qo = torch.tensor(I.taylor_green(xo, Ma=0.1))
    assert_parity(s.rhs(q), O.rhs(qo, mesh, gas), qo, mesh, gas)


def test_init_state_p15():
    from paper_1911_10966_gb300.solver import Solver
    s = Solver.box(15, 2, 1, 1, warp=0.1, seed=4, Ma=0.1, Re=1600.0)
    assert _rel(s.init_state("tgv"), I.taylor_green(s.coords, Ma=0.1)) <= 1e-14
