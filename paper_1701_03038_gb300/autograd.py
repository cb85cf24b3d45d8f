"""Differentiation through forward-backward: d log Z / d theta.

For a string x, d log Z(x) / d theta_k is the expected number of times arc k
is used, sum_t gamma_t(k) (the expected counts of Alg. 2, used for EM and
CRF-style training).  ``FstLogZ`` runs the batched forward pass in its
forward and the fused backward pass (posteriors weighted by the incoming
gradient g_b of each string) in its backward, so the gradient costs one
backward pass and no second forward.
"""
from __future__ import annotations

import torch

from .fst import Fst, Plan

__all__ = ["FstLogZ", "log_z", "LogZModule"]


class FstLogZ(torch.autograd.Function):
    """log Z of every string of ``plan`` as a function of the arc log-weights.

    forward(theta [A] float32 CUDA, fst, plan) -> log Z [B] float64.
    ``plan`` must be a single-wave plan of ``fst`` (flags PLAN_SINGLE_WAVE)."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, fst: Fst, plan: Plan):
        fst.set_weights(theta.detach(), "log")
        plan.forward()
        ctx.plan = plan
        ctx.num_arcs = fst.num_arcs
        return plan.logz[:plan.B].clone()

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        plan = ctx.plan
        g = grad_out.detach().to(torch.float32).contiguous()
        plan.backward(g)
        return plan.counts[:ctx.num_arcs].clone(), None, None


def log_z(theta: torch.Tensor, fst: Fst, plan: Plan) -> torch.Tensor:
    """Autograd-aware log Z [B] (see FstLogZ)."""
    return FstLogZ.apply(theta, fst, plan)


class LogZModule(torch.nn.Module):
    """Arc log-weights as a parameter; forward(plan) returns log Z per string.

    A CRF/HMM-style training step minimises a loss of log Z (for example the
    negative log-likelihood log Z(x) - score(x, y)); its gradient with
    respect to the weights comes from the fused backward pass."""

    def __init__(self, fst: Fst, theta0: torch.Tensor):
        super().__init__()
        self.fst = fst
        self.theta = torch.nn.Parameter(theta0.detach().to(device=fst.device, dtype=torch.float32).clone())

    def forward(self, plan: Plan) -> torch.Tensor:
        return FstLogZ.apply(self.theta, self.fst, plan)
