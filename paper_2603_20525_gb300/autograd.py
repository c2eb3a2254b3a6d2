"""Differentiable rollout cost and constraint margin, and gradient refinement
of plan candidates.

`RolloutCost` wraps the hand-written adjoint (atp_grad) in a
torch.autograd.Function: its forward returns each candidate's cost J and its
backward returns dJ/dctrl from the same launch.  `RolloutMargin` does the
same for each candidate's ESM margin, the minimum of U_ESM over its
trajectory (atp_grad_margin).  `refine` runs projected gradient descent on a
set of candidates with the library's step kernels (atp_refine_*): the
steering rate kept inside its limit, a step accepted per candidate only when
its cost decreases.  PyTorch holds the buffers; every step of the arithmetic
runs in the library's kernels.
"""
from __future__ import annotations

import torch


class RolloutCost(torch.autograd.Function):
    """J = RolloutCost.apply(ctrl [H, K, 2], planner, veh, cost, terrain, x0, dt, n_sub, ckpt)."""

    @staticmethod
    def forward(ctx, ctrl, planner, veh, cst, terrain, x0, dt, n_sub=0, ckpt=10):
        J, G = planner.grad(veh, cst, terrain, x0, ctrl.detach().contiguous(), dt, n_sub, ckpt)
        ctx.save_for_backward(G)
        return J

    @staticmethod
    def backward(ctx, gJ):
        (G,) = ctx.saved_tensors
        return (gJ[None, :, None] * G,) + (None,) * 8


class RolloutMargin(torch.autograd.Function):
    """m = RolloutMargin.apply(ctrl [H, K, 2], planner, veh, cost, terrain, x0, dt, n_sub, ckpt):
    each candidate's min U_ESM over its trajectory, differentiable in ctrl."""

    @staticmethod
    def forward(ctx, ctrl, planner, veh, cst, terrain, x0, dt, n_sub=0, ckpt=10):
        m, G = planner.grad(veh, cst, terrain, x0, ctrl.detach().contiguous(), dt, n_sub, ckpt,
                            objective="margin")
        ctx.save_for_backward(G)
        return m

    @staticmethod
    def backward(ctx, gm):
        (G,) = ctx.saved_tensors
        return (gm[None, :, None] * G,) + (None,) * 8


def refine(planner, veh, cst, terrain, x0, ctrl, dt, n_sub=0, iters=10, step=0.05, ckpt=10):
    """Projected gradient descent on candidates ctrl [H, K, 2] (CUDA).  The
    step of each candidate starts at `step` / max|dJ/dctrl|, grows by 1.5
    after an accepted step and halves after a rejected one.  Returns the
    refined controls and the cost history [iters + 1, K]."""
    rate_max = float(veh["delta_rate_max"])
    ctrl = ctrl.detach().clone().contiguous()
    J, G = planner.grad(veh, cst, terrain, x0, ctrl, dt, n_sub, ckpt)
    eta = torch.empty_like(J)
    trial = torch.empty_like(ctrl)
    planner.refine_init(G, step, eta)
    hist = [J.clone()]
    for _ in range(iters):
        planner.refine_trial(ctrl, G, eta, rate_max, trial)
        Jt, Gt = planner.grad(veh, cst, terrain, x0, trial, dt, n_sub, ckpt)
        planner.refine_accept(trial, Jt, Gt, ctrl, J, G, eta)
        hist.append(J.clone())
    return ctrl, torch.stack(hist)
