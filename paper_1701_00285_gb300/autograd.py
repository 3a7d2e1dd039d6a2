"""torch.autograd.Function around the library's BLUP loss and its adjoint
gradient (mlb_grad): the loss of held-out predictions as a differentiable
function of log(rho) and log(nugget).  Forward and backward run in the
library's CUDA kernels; this module only moves scalars."""
from __future__ import annotations

import math

import torch

from .binding import Context


class HeldOutLoss(torch.autograd.Function):
    """loss = mean_k (Y-hat_k - y_k)^2 with Y-hat the multilevel BLUP at the
    held-out points, as a function of (log rho, log nugget)."""

    @staticmethod
    def forward(ctx_, log_rho: torch.Tensor, log_nugget: torch.Tensor, problem: dict):
        c: Context = problem["context"]
        rho = math.exp(float(log_rho))
        nug = math.exp(float(log_nugget))
        c.assemble(problem["nu"], rho, nug, problem.get("tau_factor", math.inf))
        c.solve(problem["Z"])
        loss, g_rho, g_nug = c.grad(problem["targets"], problem["y"])
        ctx_.save_for_backward(torch.tensor([g_rho, g_nug], dtype=torch.float64))
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx_, grad_out):
        (g,) = ctx_.saved_tensors
        return grad_out * g[0], grad_out * g[1], None


def held_out_loss(log_rho: torch.Tensor, log_nugget: torch.Tensor, problem: dict) -> torch.Tensor:
    return HeldOutLoss.apply(log_rho, log_nugget, problem)
