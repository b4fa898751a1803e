"""torch.autograd.Function over the hand-written adjoint (ctm_grad).

Forward runs warm-up steps (detached), k tracked CTMRG steps with checkpoints
and the energy; backward returns the gradient that ctm_grad computed
alongside, scaled by the incoming cotangent.  Both run in libctm's kernels.
"""
from __future__ import annotations

import torch

from . import binding


class CTMEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, chi, h, warmup, k_tracked, precision):
        ctm = binding.CTM(A.detach(), chi, precision=precision)
        try:
            E, dA = ctm.ctm_grad(h, warmup=warmup, k_tracked=k_tracked)
        finally:
            ctm.close()
        ctx.save_for_backward(dA)
        return torch.tensor(E, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(ctx, gE):
        (dA,) = ctx.saved_tensors
        return gE * dA, None, None, None, None, None


def ctm_energy(A, chi, h, warmup=10, k_tracked=24, precision="fp64"):
    """E_site(A) with the environment from CTMRG; differentiable w.r.t. A."""
    return CTMEnergy.apply(A, chi, h, warmup, k_tracked, precision)
