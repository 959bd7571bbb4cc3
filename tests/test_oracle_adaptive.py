"""Pins of the oracle's adaptive Dormand-Prince 5(4) integrator against properties fixed by the
mathematics: the order conditions of the embedded weights, the O(dt^5) size of the error estimate,
the fixed point of the H211b filter in closed form, the limiter, tolerance proportionality and exact
landing on the end time, and agreement with the fixed-step DP5 update."""
import math

import torch

from oracle import esdc_oracle as O

F64 = torch.float64


def _tableau():
    A = torch.zeros(7, 7, dtype=F64)
    for i, row in enumerate(O.DP5_A):
        for j, a in enumerate(row):
            A[i, j] = a
    for j, b in enumerate(O.DP5_B):
        A[6, j] = b                     # first-same-as-last: stage 7 is the new solution
    c = A.sum(dim=1)
    return A, c


def test_embedded_weights_satisfy_the_fourth_order_conditions_only():
    """The eight order conditions up to order 4 (Butcher trees) hold for bhat to round-off; the
    fifth-order bushy-tree condition fails, so bhat is the embedded 4th-order method."""
    A, c = _tableau()
    bh = torch.tensor(O.DP5_BHAT, dtype=F64)
    conds = [
        (bh.sum(), 1.0),
        (bh @ c, 1 / 2),
        (bh @ c ** 2, 1 / 3),
        (bh @ (A @ c), 1 / 6),
        (bh @ c ** 3, 1 / 4),
        (bh @ (c * (A @ c)), 1 / 8),
        (bh @ (A @ c ** 2), 1 / 12),
        (bh @ (A @ (A @ c)), 1 / 24),
    ]
    for got, want in conds:
        assert abs(float(got) - want) < 1e-14
    assert abs(float(bh @ c ** 4) - 1 / 5) > 1e-4
    # the row sums of A reproduce the stage times c of the pair
    assert torch.allclose(c[:6], torch.tensor(O.DP5_C, dtype=F64), atol=1e-15)
    assert abs(float(c[6]) - 1.0) < 1e-15


def test_error_estimate_is_fifth_order_in_dt():
    """y' = y^2, y(0) = 1: the local error estimate of one step scales like dt^5."""
    f = lambda y: y * y
    q = torch.ones(1, dtype=F64)
    errs = []
    for h in (0.02, 0.01, 0.005):
        _, _, ev = O.dp54_step(q, f(q), f, h)
        errs.append(float(ev.abs()))
    for a, b in zip(errs, errs[1:]):
        assert abs(math.log2(a / b) - 5.0) < 0.15


def test_error_norm_is_the_weighted_rms():
    """sc = atol + rtol max(|q0|, |q1|); a constant ratio e/sc = c gives c, a single nonzero ratio
    among n values gives c/sqrt(n) (a max norm would give c)."""
    q0 = torch.tensor([1.0, -2.0, 0.5, 4.0], dtype=F64)
    q1 = torch.tensor([-1.5, 1.0, 0.25, 3.0], dtype=F64)
    rtol, atol = 1e-3, 1e-4
    sc = atol + rtol * torch.tensor([1.5, 2.0, 0.5, 4.0], dtype=F64)
    assert abs(O.dp54_error_norm(q0, q1, 0.7 * sc, rtol, atol) - 0.7) < 1e-15
    e = torch.zeros(4, dtype=F64)
    e[2] = 3.0 * sc[2]
    assert abs(O.dp54_error_norm(q0, q1, e, rtol, atol) - 1.5) < 1e-15


def test_dp54_step_solution_equals_fixed_step_dp5():
    f = lambda y: torch.sin(y) - 0.3 * y
    q = torch.tensor([0.7, -1.1, 2.0], dtype=F64)
    qn, k7, _ = O.dp54_step(q, f(q), f, 0.13)
    assert torch.equal(qn, O.rk_step(q, f, 0.13, 1))
    assert torch.equal(k7, f(qn))


def test_h211b_fixed_point_and_limiter():
    """With a constant error norm c the ratio sequence of H211b converges to
    rho* = (theta/c)^(2/(k (b + 1))) (fixed point of rho = (theta/c)^(2/(b k)) rho^(-1/b)); err = theta
    gives rho = 1.  The limiter is 1 at 1 with unit slope and stays in (1 - pi/2, 1 + pi/2)."""
    for cst in (0.1, 0.5, 2.0):
        rho = 1.0
        for _ in range(200):
            rho = O.h211b_ratio(cst, cst, rho)
        want = (O.CTRL_THETA / cst) ** (2.0 / (O.DP54_K * (O.H211B_B + 1.0)))
        assert abs(rho - want) < 1e-12 * want
    assert O.h211b_ratio(O.CTRL_THETA, O.CTRL_THETA, 1.0) == 1.0
    assert O.step_limiter(1.0) == 1.0
    d = 1e-6
    assert abs((O.step_limiter(1 + d) - O.step_limiter(1 - d)) / (2 * d) - 1.0) < 1e-9
    assert 1 - math.pi / 2 < O.step_limiter(-1e9) < O.step_limiter(1e9) < 1 + math.pi / 2


def test_adaptive_linear_decay_meets_tolerance_and_lands_on_t_end():
    """y' = -y on [0, 2]: the global error follows the tolerance, the step count grows like
    tol^(-1/5), the accepted steps add up to t_end exactly, and one residual per attempted stage."""
    f = lambda y: -y
    res = {}
    for tol in (1e-6, 1e-9):
        y, st = O.rk_adaptive(torch.ones(1, dtype=F64), f, 0.0, 2.0, 0.1, tol, tol)
        err = abs(float(y) - math.exp(-2.0))
        assert err < 50 * tol
        assert abs(sum(st["accepted"]) - 2.0) < 1e-14
        assert st["rhs"] == 1 + 6 * (len(st["accepted"]) + st["rejected"])
        res[tol] = len(st["accepted"])
    ratio = res[1e-9] / res[1e-6]
    assert 1000 ** 0.2 * 0.6 < ratio < 1000 ** 0.2 * 1.6


def test_too_large_first_step_is_rejected_then_recovers():
    f = lambda y: -50.0 * (y - torch.cos(torch.tensor(0.0, dtype=F64)))
    y, st = O.rk_adaptive(torch.zeros(1, dtype=F64), f, 0.0, 1.0, 0.5, 1e-8, 1e-8)
    assert st["rejected"] >= 1
    assert abs(float(y) - (1.0 - math.exp(-50.0))) < 1e-6


def test_unphysical_trial_step_counts_as_zero_ratio():
    """A trial step so large that a stage state leaves the domain of f (here y <= 0, where f returns
    NaN) is rejected with the limiter's floor L(0) = 1 - pi/4 instead of propagating NaN."""
    f = lambda y: torch.where(y > 0, -y, torch.full_like(y, float("nan")))
    y, st = O.rk_adaptive(torch.ones(1, dtype=F64), f, 0.0, 1.0, 8.0, 1e-8, 1e-8)
    assert st["rejected"] >= 1 and abs(float(y) - math.exp(-1.0)) < 1e-6
    assert abs(O.step_limiter(0.0) - (1.0 - math.pi / 4.0)) < 1e-15


def test_zero_length_interval_takes_no_step():
    q = torch.ones(2, dtype=F64)
    y, st = O.rk_adaptive(q, lambda y: -y, 1.0, 1.0, 0.1, 1e-6, 1e-6)
    assert torch.equal(y, q) and st["accepted"] == [] and st["rejected"] == 0 and st["rhs"] == 0
