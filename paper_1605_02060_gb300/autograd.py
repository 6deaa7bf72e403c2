"""torch.autograd binding of the exact energy gradient (lddmm_energy_grad).

``LddmmEnergy.apply(v, ctx)`` returns the discrete masked-LDDMM energy (§2.4) of the velocity
field ``v`` ([T][3][nz][ny][nx] float32, CUDA) for the images held by the liblddmm context
``ctx``; its backward pass returns dE/dv, computed on the GPU by the reverse-mode sweep of the
library (the forward maps are stored, or checkpointed when the context was created with
params.flags bit 1).  All arithmetic runs in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from .lddmm import Lddmm


class LddmmEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, v: torch.Tensor, ctx: Lddmm):
        if not v.is_cuda or v.dtype != torch.float32:
            raise TypeError("v must be a float32 CUDA tensor")
        v = v.detach().contiguous()
        grad = torch.empty_like(v)
        E, _ = ctx.energy_grad(v, grad)
        fctx.save_for_backward(grad)
        return torch.tensor(E, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(fctx, gE):
        (grad,) = fctx.saved_tensors
        return gE.to(grad.dtype) * grad, None


def energy(v: torch.Tensor, ctx: Lddmm) -> torch.Tensor:
    """Differentiable energy of v (see LddmmEnergy)."""
    return LddmmEnergy.apply(v, ctx)


def batched_energy(vs, ctxs):
    """Sum of the energies of independent registrations (one context per pair)."""
    return sum(LddmmEnergy.apply(v, c) for v, c in zip(vs, ctxs))
