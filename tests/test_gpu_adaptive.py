"""Adaptive Dormand-Prince 5(4) (esdc_rk_adaptive) against the oracle's rk_adaptive on the same
seeded workloads: the same accepted and rejected steps, step sizes and final state.  The error
estimate dt sum_j (b_j - bhat_j) k_j cancels the stage derivatives down to ~1e-7 of their size, so
the residuals' rounding-level differences (~1e-13 relative) become ~1e-10 relative in the error
norm, ~5e-12 in each step-size ratio (the filter takes its 20th root) and, through the filter's
memory and the final step t_end - t, ~1e-10 in the step sizes: the tolerances below are 1e-9 for
step sizes and 1e-10 for the final state."""
import math

import pytest
import torch

from oracle import esdc_oracle as O
from tests.gpu_common import make_pair, normwise_errors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,k,Re,state,tol", [(2, (3, 3, 2), 200.0, "tgv", 1e-6),
                                              (3, (2, 2, 2), 0.0, "vortex", 1e-7)])
def test_adaptive_matches_oracle(p, k, Re, state, tol):
    box = ([-5.0] * 3, [5.0] * 3) if state == "vortex" else None
    kw = {"box": box} if box else {}
    Ma = 0.5 if state == "vortex" else 0.1
    solver, qg, mesh, gas, qo = make_pair(p, k, warp=0.1, seed=2, Re=Re, Ma=Ma, state=state, **kw)
    dt_cfl = solver.dt_cfl(qg, 0.5)
    dt0 = 4.0 * dt_cfl                  # too large on purpose: the first attempt is rejected
    t_end = 12.0 * dt_cfl
    st = solver.rk_adaptive(qg, 0.0, t_end, dt0, rtol=tol, atol=tol, max_steps=400, history=1000)
    qo_end, so = O.rk_adaptive(qo, lambda s: O.rhs(s, mesh, gas), 0.0, t_end, dt0, tol, tol, max_steps=400)
    print("gpu", {k_: v for k_, v in st.items() if k_ != "dt_history"}, "oracle accepted", len(so["accepted"]),
          "rejected", so["rejected"])
    assert st["accepted"] == len(so["accepted"]) and st["rejected"] == so["rejected"]
    assert st["rhs"] == so["rhs"] and st["rejected"] >= 1
    assert st["t"] == t_end
    for a, b in zip(st["dt_history"], so["accepted"]):
        assert abs(a - b) <= 1e-9 * b
    # the proposal after the last step comes from a step shortened to t_end - t (a difference that
    # loses ~3 digits) whose tiny error estimate is rounding-dominated: compared loosely
    assert abs(st["dt_next"] - so["dt_next"]) <= 1e-6 * so["dt_next"]
    e = normwise_errors(qg, qo_end)
    print("final state", ["%.1e" % x for x in e])
    assert max(e) <= 1e-10


def test_adaptive_edge_cases():
    """t_end = t0 takes no step and evaluates nothing; max_steps stops early and reports the time
    reached; bad arguments are rejected without touching the state."""
    from paper_1911_10966_gb300 import _native as nat
    from paper_1911_10966_gb300.solver import Solver
    solver, qg, mesh, gas, qo = make_pair(2, (2, 2, 2), Re=100.0)
    q0 = qg.clone()
    st = solver.rk_adaptive(qg, 1.0, 1.0, 1e-3)
    assert st["accepted"] == 0 and st["rejected"] == 0 and st["rhs"] == 0 and torch.equal(qg, q0)
    dt = solver.dt_cfl(qg, 0.5)
    st = solver.rk_adaptive(qg, 0.0, 100.0 * dt, dt, rtol=1e-8, atol=1e-8, max_steps=3)
    assert st["accepted"] + st["rejected"] == 3 and 0.0 < st["t"] < 100.0 * dt
    for bad in (dict(dt0=0.0), dict(dt0=-1.0), dict(rtol=0.0), dict(atol=-1.0), dict(t_end=-1.0)):
        args = dict(t0=0.0, t_end=1.0, dt0=1e-3, rtol=1e-6, atol=1e-6)
        args.update(bad)
        q1 = qg.clone()
        with pytest.raises(nat.EsdcError) as ei:
            solver.rk_adaptive(q1, args["t0"], args["t_end"], args["dt0"], rtol=args["rtol"], atol=args["atol"])
        assert ei.value.code == nat.ESDC_ERR_ARG and torch.equal(q1, qg)


def test_adaptive_fp32_mixed_follows_the_float64_integrator():
    """Float32-mixed context at a tolerance far above float32 rounding of the residual: it reaches
    t_end with the float64 integrator's accepted and rejected step counts (within one), the same step
    sizes to 1e-3, and a final state within 1e-5 of the float64 one (measured: equal step counts, 6.9e-8
relative difference of the next step proposal, 7.8e-6 in rho u3 relative to its small maximum)."""
    from paper_1911_10966_gb300.solver import Solver
    s64, q64, mesh, gas, qo = make_pair(3, (3, 3, 3), warp=0.1, seed=2, Re=400.0, Ma=0.1, state="tgv")
    s32 = Solver(3, 3, 3, 3, s64.coords, Re=400.0, Ma=0.1, precision="fp32")
    q32 = q64.clone()
    dt_cfl = s64.dt_cfl(q64, 0.5)
    t_end = 20.0 * dt_cfl
    st64 = s64.rk_adaptive(q64, 0.0, t_end, 4.0 * dt_cfl, rtol=1e-5, atol=1e-5, history=1000)
    st32 = s32.rk_adaptive(q32, 0.0, t_end, 4.0 * dt_cfl, rtol=1e-5, atol=1e-5, history=1000)
    print("fp64", {k: v for k, v in st64.items() if k != "dt_history"},
          "fp32", {k: v for k, v in st32.items() if k != "dt_history"})
    assert st32["t"] == t_end
    assert abs(st32["accepted"] - st64["accepted"]) <= 1 and abs(st32["rejected"] - st64["rejected"]) <= 1
    if st32["accepted"] == st64["accepted"]:
        for a, b in zip(st32["dt_history"], st64["dt_history"]):
            assert abs(a - b) <= 1e-3 * b
    # relative to max(|q_v|, 0.1): the Taylor-Green rho u3 starts at zero and stays small
    e = normwise_errors(q32, q64.cpu(), abs_floor=0.1)
    print("fp32 vs fp64 adaptive final state", ["%.1e" % x for x in e])
    assert max(e) <= 1e-5
