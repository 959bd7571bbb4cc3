"""torch.autograd.Function wrappers of the residual, the DP5 trajectory and the kinetic energy.

Forward passes call the library's float64 kernels; backward passes call its hand-written adjoint
kernels (esdc_rhs_vjp; esdc_rk_adjoint_stages from stored stage states, or esdc_rk_adjoint from
per-step checkpoints with stage recomputation; esdc_ke_gradient).  Nothing here differentiates
through torch operations.
"""
from __future__ import annotations

import torch


class Residual(torch.autograd.Function):
    """R(q) = dq/dt; backward: (dR/dq)^T grad_out."""

    @staticmethod
    def forward(ctx, q, solver):
        ctx.solver = solver
        ctx.save_for_backward(q)
        return solver.rhs(q.detach().contiguous())

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        return ctx.solver.rhs_vjp(q.detach().contiguous(), g.contiguous()), None


class Trajectory(torch.autograd.Function):
    """q_N after nsteps fixed DP5 steps from q_0, as a function of (q_0, mu).  mu must equal the
    solver's viscosity (it is an input only so that dL/dmu can flow back).

    stages: checkpoint granularity of the reverse sweep.  True stores the six stage states of every
    step (6 x nsteps states, no recomputation); False stores the state before each step with its
    residual (2 x nsteps states) and recomputes the stage states in the reverse sweep (four residuals
    per step), or the state alone (nsteps states, five residuals per step) when the pair does not fit
    in half of the free device memory; None picks True when the stage states fit there."""

    @staticmethod
    def forward(ctx, q0, mu, solver, dt, nsteps, stages=None):
        if abs(float(mu) - solver.mu) > 1e-15 * max(1.0, abs(solver.mu)):
            raise ValueError("mu must equal the solver's viscosity 1/Re")
        free, _ = torch.cuda.mem_get_info(q0.device)
        if stages is None:
            stages = 6 * nsteps * q0.numel() * 8 <= free // 2
        k1 = 2 * nsteps * q0.numel() * 8 <= free // 2
        q = q0.detach().clone().contiguous()
        ck = solver.rk_step_ckpt(q, dt, nsteps, stages=bool(stages), k1=k1)
        ctx.solver, ctx.dt = solver, dt
        ctx.save_for_backward(ck)
        return q

    @staticmethod
    def backward(ctx, g):
        (ck,) = ctx.saved_tensors
        lam = g.detach().clone().contiguous()
        lam, gmu = ctx.solver.rk_adjoint(ck, ctx.dt, lam)
        return lam, torch.tensor(gmu, dtype=torch.float64, device=lam.device), None, None, None, None


class KineticEnergy(torch.autograd.Function):
    """sum P J rho|u|^2/2 (a 0-d float64 tensor on the solver's device)."""

    @staticmethod
    def forward(ctx, q, solver):
        ctx.solver = solver
        ctx.save_for_backward(q)
        ke = solver.budgets(q.detach().contiguous())[1]
        return torch.tensor(ke, dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(ctx, g):
        (q,) = ctx.saved_tensors
        return g * ctx.solver.ke_gradient(q.detach().contiguous()), None
