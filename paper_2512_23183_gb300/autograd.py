"""torch.autograd.Function around the library's adjoint gradient.

``energy(params, n, gates, terms)`` returns E(theta) = <psi(theta)|H|psi(theta)>
as a 0-d float64 tensor whose backward pass uses the gradient computed by
lq_adjoint_grad (reverse-mode differentiation through the circuit).
"""
import numpy as np
import torch


class AdjointEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, n, gates, terms, device):
        from . import adjoint_grad

        p = params.detach().to("cpu", torch.float64).numpy()
        e, g = adjoint_grad(n, gates, p, terms, device=device)
        ctx.save_for_backward(torch.from_numpy(np.asarray(g, np.float64)).to(params.device))
        return torch.tensor(e, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None


def energy(params, n, gates, terms, device="cuda"):
    """Differentiable E(theta); params is a 1-d float64 tensor."""
    return AdjointEnergy.apply(params, n, gates, terms, device)
