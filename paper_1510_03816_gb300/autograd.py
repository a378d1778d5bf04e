"""torch.autograd bridge of the inexact-matching energy (Sec. 6, Eq. inexact-E).

E(p0) = 1/2 p0^T G(X) p0 + lambda/2 ||Q(1) - Y||^2 is evaluated, together with
its exact discrete-adjoint gradient dE/dp0, by one ep_adjoint call in the
forward pass; backward scales the stored gradient.  X and Y are treated as
constants (no gradient).  Nothing here computes any part of the method.
"""
from __future__ import annotations

import torch

from . import ep


class EPInexactEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, p0, Y, prm, lam, ckpt_every):
        E, g = ep.adjoint(X.detach(), p0.detach(), Y.detach(), prm, lam, ckpt_every)
        ctx.save_for_backward(g)
        return torch.tensor(E, dtype=torch.float64, device=p0.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return None, grad_out * g, None, None, None, None


def inexact_energy(X, p0, Y, prm: ep.Params, lam: float, ckpt_every: int = 10) -> torch.Tensor:
    """Differentiable E(p0); ``backward()`` fills ``p0.grad`` with dE/dp0 (ep_adjoint)."""
    return EPInexactEnergy.apply(X, p0, Y, prm, float(lam), int(ckpt_every))
