"""Differentiable QFactor cost for PyTorch.

QFactorCost.apply(gates, target, locations) returns, for every gate set s,
cost_s = 1 - |Tr(V^dagger C(gates_s))| / N (Sec. II, Delta).  Because every
gate enters Tr(V^dagger C) linearly through its environment (Sec. III,
Tr(V^dagger U) = Tr(E u_k)), one adjoint walk of the circuit tensor on the GPU
(qf_cost_grad) gives the cost and the gradient of all p gates at once; the
forward pass runs it when the gates require a gradient and keeps the result
for backward.
"""
from __future__ import annotations

import torch

from . import api


class QFactorCost(torch.autograd.Function):
    """``locations`` of qubit pairs take gates (S, p, 4, 4) or (p, 4, 4);
    locations with 3- or 4-qubit gates take the concatenated layout (S, E)
    or (E,) (qf_cost_grad_k)."""

    @staticmethod
    def forward(ctx, gates, target, locations):
        pairs = api._is_pairs(locations)
        single = gates.dim() == (3 if pairs else 1)
        if ctx.needs_input_grad[0]:
            if pairs:
                c, g = api.cost_grad(target, locations, gates.detach())
            else:
                c, g = api.cost_grad_k(target, locations, gates.detach())
            ctx.save_for_backward(g)
        else:
            if pairs:
                c = api.costs(target, locations, gates.detach())
                if single:
                    c = c[0]
            else:
                c = api.cost_and_env_k(target, locations, gates.detach())[0]
        ctx.single = single
        return torch.as_tensor(c, dtype=torch.float64, device=gates.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        scale = grad_out.to(g.device, torch.float64)
        if ctx.single:
            return g * scale, None, None
        return g * scale.reshape((-1,) + (1,) * (g.dim() - 1)), None, None


def qfactor_cost(gates, target, locations):
    """Functional form of QFactorCost."""
    return QFactorCost.apply(gates, target, locations)
