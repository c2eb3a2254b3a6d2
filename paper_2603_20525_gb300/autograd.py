"""Differentiable rollout cost and gradient refinement of plan candidates.

`RolloutCost` wraps the hand-written adjoint (atp_grad) in a
torch.autograd.Function: its forward returns each candidate's cost J and its
backward returns dJ/dctrl from the same launch.  `refine` runs projected
gradient descent on a set of candidates (the steering rate kept inside its
limit), accepting a step per candidate only when its cost decreases.
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


def refine(planner, veh, cst, terrain, x0, ctrl, dt, n_sub=0, iters=10, step=0.05, ckpt=10):
    """Projected gradient descent on candidates ctrl [H, K, 2] (CUDA).  The
    step of each candidate starts at `step` / max|dJ/dctrl|, grows by 1.5
    after an accepted step and halves after a rejected one.  Returns the
    refined controls and the cost history [iters + 1, K]."""
    rate_max = float(veh["delta_rate_max"])
    ctrl = ctrl.detach().clone().contiguous()
    J, G = planner.grad(veh, cst, terrain, x0, ctrl, dt, n_sub, ckpt)
    eta = step / (G.abs().amax(dim=(0, 2)) + 1e-12)
    hist = [J.clone()]
    for _ in range(iters):
        trial = ctrl - eta[None, :, None] * G
        trial[..., 0].clamp_(-rate_max, rate_max)
        trial = trial.contiguous()
        Jt, Gt = planner.grad(veh, cst, terrain, x0, trial, dt, n_sub, ckpt)
        ok = torch.isfinite(Jt) & (Jt < J)
        ctrl = torch.where(ok[None, :, None], trial, ctrl)
        G = torch.where(ok[None, :, None], Gt, G)
        J = torch.where(ok, Jt, J)
        eta = torch.where(ok, eta * 1.5, eta * 0.5)
        hist.append(J.clone())
    return ctrl, torch.stack(hist)
