"""The allocation-free budget reduction (esdc_budgets_noalloc) against the context-based one.

Callers such as code running while a stream is being captured, or hosts that hand all device memory
to their own allocator at start-up, cannot call cudaMalloc; esdc_budgets_noalloc serves them from a
static device array.  This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It builds everything it needs itself, so it passes
alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1911_10966_gb300 import _native as nat
from tests.gpu_common import make_pair

pytestmark = pytest.mark.gpu


def _noalloc(solver, w, J_dev, q, dq, out):
    L = nat.lib()
    code = L.esdc_budgets_noalloc(solver.N, solver.K, solver.gamma, w.ctypes.data, q.data_ptr(),
                                  dq.data_ptr() if dq is not None else None, J_dev.data_ptr(), out.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    nat.check(code, "esdc_budgets_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


def _close(a, b, rel):
    return abs(a - b) <= rel * max(abs(b), 1e-300)


def test_budgets_noalloc_matches_context_budgets_twice():
    solver, q1, _, _, _ = make_pair(4, (6, 5, 4), warp=0.1, seed=2, Re=1600.0, noise=1e-2)
    w = np.zeros(solver.N)
    xi = np.zeros(solver.N)
    nat.check(nat.lib().esdc_lgl(solver.p, xi.ctypes.data, w.ctypes.data), "esdc_lgl")
    J, _ = solver.geometry()
    J_dev = torch.as_tensor(np.ascontiguousarray(J), device=q1.device)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=q1.device)
    # second input: a different state, so stale scratch from the first call would show
    q2 = q1.clone()
    q2[:, 4] *= 1.01
    for q in (q1, q2):
        dq = solver.rhs(q)
        ref = solver.budgets(q, dq)
        got = _noalloc(solver, w, J_dev, q, dq, out)
        # same tolerances as the context budget tests: 1e-13 relative for S and KE, and for the
        # rates 1e-12 relative to their size (different but fixed summation orders)
        assert got[4] == 0.0
        assert _close(got[0], ref[0], 1e-13) and _close(got[1], ref[1], 1e-13), (got, ref)
        assert _close(got[2], ref[2], 1e-12) and _close(got[3], ref[3], 1e-12), (got, ref)
        got0 = _noalloc(solver, w, J_dev, q, None, out)
        assert _close(got0[0], ref[0], 1e-13) and got0[2] == 0.0 and got0[3] == 0.0


def test_budgets_noalloc_rejects_oversized_input():
    solver, q, _, _, _ = make_pair(2, (2, 2, 2), Re=0.0)
    w = np.ones(3)
    out = torch.zeros(5, dtype=torch.float64, device=q.device)
    L = nat.lib()
    code = L.esdc_budgets_noalloc(8, 10 ** 6, 1.4, w.ctypes.data, q.data_ptr(), None, q.data_ptr(),
                                  out.data_ptr(), None)
    assert code == nat.ESDC_ERR_ARG
    assert b"static scratch limit" in L.esdc_last_error()


def test_budgets_noalloc_counts_nonphysical_nodes_like_context_budgets():
    """A negative density and a non-finite residual entry: both reductions skip the non-physical node's
    entropy and energy terms and count two bad nodes; their sums agree on the remaining nodes."""
    solver, q, _, _, _ = make_pair(3, (4, 3, 2), warp=0.1, seed=3, Re=1600.0, noise=1e-2)
    w = np.zeros(solver.N)
    xi = np.zeros(solver.N)
    nat.check(nat.lib().esdc_lgl(solver.p, xi.ctypes.data, w.ctypes.data), "esdc_lgl")
    J, _ = solver.geometry()
    J_dev = torch.as_tensor(np.ascontiguousarray(J), device=q.device)
    dq = solver.rhs(q)
    bad = q.clone()
    bad[2, 0, 1, 2, 0] = -0.5
    dq[5, 3, 0, 1, 1] = float("nan")
    ctx = torch.full((5,), float("nan"), dtype=torch.float64, device=q.device)
    solver.budgets_async(bad, ctx)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=q.device)
    got = _noalloc(solver, w, J_dev, bad, None, out)
    ref = ctx.cpu().numpy()
    assert got[4] == ref[4] == 1.0
    assert _close(got[0], ref[0], 1e-13) and _close(got[1], ref[1], 1e-13), (got, ref)
    solver.budgets_async(bad, ctx, dq)
    got = _noalloc(solver, w, J_dev, bad, dq, out)
    ref = ctx.cpu().numpy()
    assert got[4] == ref[4] == 2.0
    assert _close(got[0], ref[0], 1e-13) and _close(got[1], ref[1], 1e-13), (got, ref)
    assert np.isnan(got[2]) and np.isnan(ref[2]) and np.isnan(got[3]) and np.isnan(ref[3])
    # the same input once more after a clean call: nothing of the earlier call leaks into the sums
    _noalloc(solver, w, J_dev, q, solver.rhs(q), out)
    got2 = _noalloc(solver, w, J_dev, bad, None, out)
    assert got2[4] == 1.0 and _close(got2[1], got[1], 1e-13)
