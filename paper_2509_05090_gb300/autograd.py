"""torch.autograd.Function over the hand-written adjoint (ctm_grad).

Forward: warm-up plus k tracked CTMRG steps from the environment the context
holds, then the energy -- no gradient work.  Backward: the same steps again from
the saved starting environment through ctm_grad, which checkpoints them and runs
the adjoint; the gradient is scaled by the incoming cotangent.  One library
context per (shape, chi, precision, device) is kept between calls: a new site
tensor is swapped in with ctm_set_site and the previous environment is the warm
start of the next call (Sec. II.D).  All of it runs in libctm's kernels.
"""
from __future__ import annotations

import torch

from . import binding

_CONTEXTS = {}


def _context(A, chi, precision, n_split):
    dev = torch.cuda.current_device()
    key = (tuple(A.shape), int(chi), precision, int(n_split), dev)
    ctm = _CONTEXTS.get(key)
    if ctm is None:
        ctm = binding.CTM(A, chi, precision=precision, n_split=n_split)
        _CONTEXTS[key] = ctm
    elif ctm._A is not A:
        ctm.ctm_set_site(A)
    return ctm


def release_contexts():
    """Destroy the cached library contexts (their workspaces go back to torch)."""
    for ctm in _CONTEXTS.values():
        ctm.close()
    _CONTEXTS.clear()


class CTMEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, chi, h, warmup, k_tracked, precision, n_split):
        Ad = A.detach().to(device="cuda", dtype=torch.float64).contiguous()
        ctm = _context(Ad, chi, precision, n_split)
        env0 = ctm.ctm_get_env()
        ctm.ctm_step(warmup + k_tracked, want_delta=False)
        _, E, _ = ctm.ctm_energy(h)
        ctx.save_for_backward(Ad)
        ctx.env0 = env0
        ctx.cfg = (chi, h, warmup, k_tracked, precision, n_split)
        ctx.a_device, ctx.a_dtype = A.device, A.dtype
        return torch.tensor(E, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(ctx, gE):
        (Ad,) = ctx.saved_tensors
        chi, h, warmup, k_tracked, precision, n_split = ctx.cfg
        ctm = _context(Ad, chi, precision, n_split)
        ctm.ctm_set_env(*ctx.env0)
        _, dA = ctm.ctm_grad(h, warmup=warmup, k_tracked=k_tracked)
        g = gE.to(device=dA.device, dtype=torch.float64) * dA
        return g.to(device=ctx.a_device, dtype=ctx.a_dtype), None, None, None, None, None, None


def ctm_energy(A, chi, h, warmup=10, k_tracked=24, precision="fp64", n_split=5):
    """E_site(A) with the environment from CTMRG; differentiable w.r.t. A."""
    return CTMEnergy.apply(A, chi, h, warmup, k_tracked, precision, n_split)
