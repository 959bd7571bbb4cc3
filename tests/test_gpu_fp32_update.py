"""The float64 kernels of the mixed-precision step, checked bit for bit: the float32 shadow state
dq = float(q - q_ref) (round to nearest even, on every kind of value: zeros, results in the float32
subnormal range, overflow, NaN, halfway cases), and the solution update q + sum_j c_j k_j accumulated
in float64 in stage order with fused multiply-adds, replayed exactly with rational arithmetic."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DP5_B = [35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0]


def _solver():
    from paper_1911_10966_gb300.solver import Solver
    return Solver.box(2, 3, 2, 2, warp=0.1, seed=1, Ma=0.1, Re=1600.0, precision="fp32")


def _ws_views(s, n):
    sub = (n * 4 + 255) // 256 * 256
    ws = s._ws
    k = [ws[j * sub:j * sub + n * 4].view(torch.float32) for j in range(6)]
    base = ws[6 * sub:6 * sub + n * 4].view(torch.float32)
    return k, base


def _ref(s, q):
    R = 1.0 / (s.gamma * s.Ma * s.Ma)
    E0 = R / (s.gamma - 1.0)
    ref = torch.zeros_like(q)
    ref[:, 0] = 1.0
    ref[:, 4] = E0
    return ref


def test_shadow_state_rounds_like_the_hardware_on_special_values():
    s = _solver()
    q = s.init_state("tgv")
    n = q.numel()
    ref = _ref(s, q)
    flat = q.view(-1)
    g = torch.Generator().manual_seed(3)
    special = [0.0, -0.0, 1e-40, -3e-39, 1e-45, 2.0 ** -149 * 1.5, 2.0 ** -126, 3.5e38, -1e39, 1e300,
               float("inf"), float("-inf"), float("nan"), 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24,
               1.0 + 2.0 ** -24 + 2.0 ** -40, (1 + 2.0 ** -23) * 2.0 ** -127]
    # momentum entries (no reference value subtracted) take the special values directly
    mom = torch.arange(n).view(q.shape)[:, 1:4].reshape(-1)
    pick = mom[torch.randperm(mom.numel(), generator=g)[:len(special)]]
    flat[pick.to(flat.device)] = torch.tensor(special, dtype=torch.float64, device=flat.device)
    s.rk_step(q, 0.0, 0)                       # zero steps: only the shadow state is formed
    torch.cuda.synchronize()
    _, base = _ws_views(s, n)
    want = (q - ref).float().view(-1)
    got = base.clone()
    same = (got.view(torch.int32) == want.view(torch.int32)) | (torch.isnan(got) & torch.isnan(want))
    assert bool(same.all()), int((~same).sum())


def test_update_is_the_float64_fma_chain_of_the_stage_derivatives():
    s = _solver()
    q = s.init_state("tgv")
    n = q.numel()
    dt = s.dt_cfl(q, 0.5)
    q0 = q.clone()
    s.rk_step(q, dt, 1)
    torch.cuda.synchronize()
    k, _ = _ws_views(s, n)
    coef = [dt * b for b in DP5_B if b != 0.0]
    kk = [k[j].cpu().numpy() for j in range(6) if DP5_B[j] != 0.0]
    a = q0.view(-1).cpu().numpy()
    got = q.view(-1).cpu().numpy()
    idx = np.random.default_rng(5).choice(n, 1500, replace=False)
    for i in idx:
        inc = 0.0
        for c, kj in zip(coef, kk):
            kv = float(kj[i])
            inc = float(Fraction(c) * Fraction(kv) + Fraction(inc))      # fma: one rounding
        want = a[i] + inc
        assert got[i] == want or (math.isnan(got[i]) and math.isnan(want)), (i, got[i], want)
