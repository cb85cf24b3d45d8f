"""Differentiation through forward-backward: d log Z / d theta.

For a string x, d log Z(x) / d theta_k is the expected number of times arc k
is used, sum_t gamma_t(k) (the expected counts of Alg. 2, used for EM and
CRF-style training).  ``FstLogZ`` runs the batched forward pass in its
forward and the fused backward pass (posteriors weighted by the incoming
gradient g_b of each string) in its backward, so the gradient costs one
backward pass and no second forward.  The start and final log-weights may
be differentiated too: d log Z / d (start log-weight of q) is the
probability that the path starts in q, and likewise for the final state.
"""
from __future__ import annotations

import torch

from .fst import Fst, Plan

__all__ = ["FstLogZ", "log_z", "LogZModule", "crf_nll", "CrfModule"]


class FstLogZ(torch.autograd.Function):
    """log Z of every string of ``plan`` as a function of the arc log-weights
    and, optionally, of the start and final log-weights.

    forward(theta [A], fst, plan, theta_s [Q] or None, theta_f [Q] or None)
    -> log Z [B] float64 (weights float32 CUDA; None leaves the FST's own).
    ``plan`` must be a single-wave plan of ``fst`` (flags PLAN_SINGLE_WAVE)."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, fst: Fst, plan: Plan, theta_s=None, theta_f=None):
        fst.set_weights(theta.detach(), "log")
        if theta_s is not None or theta_f is not None:
            fst.set_state_weights(None if theta_s is None else theta_s.detach(),
                                  None if theta_f is None else theta_f.detach(), "log")
        plan.forward()
        ctx.plan = plan
        ctx.num_arcs = fst.num_arcs
        ctx.num_states = fst.num_states
        ctx.states = (theta_s is not None, theta_f is not None)
        return plan.logz[:plan.B].clone()

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        plan = ctx.plan
        g = grad_out.detach().to(torch.float32).contiguous()
        plan.backward(g, states=any(ctx.states))
        gs = plan.start_counts[:ctx.num_states].clone() if ctx.states[0] else None
        gf = plan.final_counts[:ctx.num_states].clone() if ctx.states[1] else None
        return plan.counts[:ctx.num_arcs].clone(), None, None, gs, gf


def log_z(theta: torch.Tensor, fst: Fst, plan: Plan, theta_s=None, theta_f=None) -> torch.Tensor:
    """Autograd-aware log Z [B] (see FstLogZ)."""
    return FstLogZ.apply(theta, fst, plan, theta_s, theta_f)


class LogZModule(torch.nn.Module):
    """Arc log-weights as a parameter; forward(plan) returns log Z per string.

    A CRF/HMM-style training step minimises a loss of log Z (for example the
    negative log-likelihood log Z(x) - score(x, y)); its gradient with
    respect to the weights comes from the fused backward pass."""

    def __init__(self, fst: Fst, theta0: torch.Tensor, theta_s0: torch.Tensor | None = None,
                 theta_f0: torch.Tensor | None = None):
        super().__init__()
        self.fst = fst

        def param(t):
            return None if t is None else torch.nn.Parameter(
                t.detach().to(device=fst.device, dtype=torch.float32).clone())
        self.theta = param(theta0)
        self.theta_s = param(theta_s0)
        self.theta_f = param(theta_f0)

    def forward(self, plan: Plan) -> torch.Tensor:
        return FstLogZ.apply(self.theta, self.fst, plan, self.theta_s, self.theta_f)


def crf_nll(theta: torch.Tensor, fst: Fst, plan_x: Plan, clamped: Fst, plan_xy: Plan) -> torch.Tensor:
    """Conditional negative log-likelihood -log p(y_b | x_b) = log Z(x_b) -
    log Z(x_b, y_b) of every string pair, differentiable in the arc
    log-weights: its gradient is the expected counts given x minus the
    expected counts given x and y.  ``plan_x`` is a single-wave plan of
    ``fst`` on the inputs x_b; ``plan_xy`` one of ``clamped``
    (``fst.clamped()``) on the pair strings ``clamped.clamp(x_b, y_b)``, in
    the same string order."""
    return FstLogZ.apply(theta, fst, plan_x, None, None) - FstLogZ.apply(theta, clamped, plan_xy, None, None)


class CrfModule(torch.nn.Module):
    """Arc log-weights as a parameter of a conditional (CRF-style) model of
    output strings given input strings; forward(plan_x, plan_xy) returns
    -log p(y_b | x_b) per string (see crf_nll).  The clamped FST shares the
    weights (it is rebuilt from the FST's arcs once)."""

    def __init__(self, fst: Fst, theta0: torch.Tensor):
        super().__init__()
        self.fst = fst
        self.clamped = fst.clamped()
        self.theta = torch.nn.Parameter(theta0.detach().to(device=fst.device, dtype=torch.float32).clone())

    def forward(self, plan_x: Plan, plan_xy: Plan) -> torch.Tensor:
        return crf_nll(self.theta, self.fst, plan_x, self.clamped, plan_xy)
