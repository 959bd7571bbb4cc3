"""Multi-step esdc_rk_step replays one DP5 step captured as a CUDA graph: the result equals, bit for bit,
the same number of single-step calls (direct launches), in float64 and float32-mixed contexts, and the
graph is rebuilt when the step size changes."""
import pytest
import torch

from tests.gpu_common import make_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_equals_direct_steps(precision):
    solver, qg, mesh, gas, qo = make_pair(3, (3, 2, 2), warp=0.1, seed=2, Re=800.0, noise=1e-2,
                                          precision=precision)
    dt = solver.dt_cfl(qg, 0.5)
    qa, qb = qg.clone(), qg.clone()
    solver.rk_step(qa, dt, 4)                 # graph path
    for _ in range(4):
        solver.rk_step(qb, dt, 1)             # direct launches
    assert torch.equal(qa, qb)
    solver.rk_step(qa, 0.5 * dt, 3)           # new step size: recaptured
    for _ in range(3):
        solver.rk_step(qb, 0.5 * dt, 1)
    assert torch.equal(qa, qb)
    solver.profile(True)                      # profiled calls launch directly
    solver.rk_step(qa, dt, 2)
    solver.profile_read()
    solver.profile(False)
    for _ in range(2):
        solver.rk_step(qb, dt, 1)
    assert torch.equal(qa, qb)
