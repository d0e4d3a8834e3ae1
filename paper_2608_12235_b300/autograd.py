"""torch.autograd binding of the fused energy/gradient kernel.

    E = RcpEnergy.apply(x, kappa, packing, mu)

x is an (N, d) float64 CUDA tensor, kappa a 0-d float64 CUDA tensor, packing
an rcp.Packing (its diameters, box and precision), mu the growth weight of
Eq. energy.  The forward is one pass of the fused pair kernel, which yields E
together with dE/dx and dE/dkappa; the hand-written backward scales those by
the incoming gradient.  Everything runs on torch's current CUDA stream; there
is no CPU path.
"""
from __future__ import annotations

import torch

from . import rcp


class RcpEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, kappa, packing, mu):
        if not (x.is_cuda and kappa.is_cuda):
            raise ValueError("RcpEnergy needs CUDA tensors")
        if x.dtype != torch.float64 or kappa.dtype != torch.float64 or x.shape != (packing.n, packing.d):
            raise ValueError("x must be float64 (N, d) and kappa a float64 scalar")
        x = x.contiguous()
        kappa = kappa.reshape(1).contiguous()
        rcp.rcp_set_stream(packing.h, rcp.torch_stream(x.device))
        E = torch.empty(1, dtype=torch.float64, device=x.device)
        dk = torch.empty(1, dtype=torch.float64, device=x.device)
        g = torch.empty_like(x)
        rcp.rcp_energy_grad_at(packing.h, x, kappa, float(mu), E, g, dk, None)
        ctx.save_for_backward(g, dk)
        return E.reshape(())

    @staticmethod
    def backward(ctx, gE):
        g, dk = ctx.saved_tensors
        return gE * g, (gE * dk).reshape(()), None, None


def energy(x, kappa, packing, mu: float = 0.0):
    """Eq. energy with autograd support (see RcpEnergy)."""
    return RcpEnergy.apply(x, kappa, packing, mu)
