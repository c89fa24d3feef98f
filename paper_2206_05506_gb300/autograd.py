"""Differentiable estimator for end-to-end pilot and receiver optimisation.

The pilot is relaxed to p = tanh(theta), theta in R^N.  Forward and backward both run in
the library's kernels (the tanh and its derivative included):

    H = (1/N) Y P(tanh theta)                              pnce_estimate_real_pilot
    dLoss/dY     = (1/N) G P^T                             pnce_backward
    dLoss/dtheta = (1/N) sum Re(conj(G) Y[(q + j) mod N]) (1 - tanh^2 theta)

G is dLoss/dRe(H) + i dLoss/dIm(H), which is the gradient PyTorch hands to backward()
for a complex output.  The estimator's arithmetic is the same FP32 correlation as the
plain path; only the pilot became a parameter.
"""
from __future__ import annotations

import torch

from . import backward as _backward
from . import estimate_real_pilot as _forward


class RelaxedPilotCorrelation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y: torch.Tensor, theta: torch.Tensor, K: int, L: int):
        Y = Y.contiguous()
        theta = theta.contiguous()
        H = _forward(Y, theta, K, L, pilot_map="tanh")
        ctx.save_for_backward(Y, theta)
        ctx.K, ctx.L = K, L
        return H

    @staticmethod
    def backward(ctx, G: torch.Tensor):
        Y, theta = ctx.saved_tensors
        need_y, need_t = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_y or need_t):
            return None, None, None, None
        dY, dtheta = _backward(theta, Y, G.contiguous(), ctx.K, ctx.L, need_dY=need_y,
                               need_dp=need_t, pilot_map="tanh")
        return dY, dtheta, None, None


def relaxed_estimate(Y: torch.Tensor, theta: torch.Tensor, K: int, L: int) -> torch.Tensor:
    """H[F, M, K, L] for received blocks Y[F, M, N] and pilot tanh(theta), differentiable."""
    return RelaxedPilotCorrelation.apply(Y, theta, K, L)
