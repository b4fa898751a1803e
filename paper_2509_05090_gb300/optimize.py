"""Variational optimisation of the site tensor (Sec. II.D).

The energy per site E(A) of the C3v-symmetric iPEPS is minimised with L-BFGS
(torch.optim.LBFGS) over the raw site tensor A.  Each evaluation runs CTMRG in
libctm through the differentiable energy of autograd.py: `warmup` steps, then
`k_tracked` steps whose adjoint gives dE/dA (ctm_grad).  The library context and
its environment persist between evaluations, so every evaluation starts from the
environment of the previous trial tensor.  A run at a larger bond dimension is
started from a converged smaller-D tensor padded with a small seeded random
perturbation (pad_site_tensor).
"""
from __future__ import annotations

import numpy as np
import torch

from . import autograd


def pad_site_tensor(A, D_new: int, eps: float, seed: int) -> np.ndarray:
    """A[s, i, j, k] (bond D) embedded in bond D_new: the old entries are kept, every new
    entry is eps * uniform[-1, 1] from default_rng(seed) (Sec. II.D's padded start)."""
    A = np.asarray(A.detach().cpu().numpy() if torch.is_tensor(A) else A, dtype=np.float64)
    d, D = A.shape[0], A.shape[1]
    if D_new < D:
        raise ValueError("D_new must not be smaller than D")
    rng = np.random.default_rng(seed)
    out = eps * rng.uniform(-1.0, 1.0, size=(d, D_new, D_new, D_new))
    out[:, :D, :D, :D] = A
    return out


def optimize(A0, chi: int, h, steps: int = 20, warmup: int = 10, k_tracked: int = 10,
             precision: str = "fp64", n_split: int = 5, lr: float = 1.0, history_size: int = 10,
             callback=None):
    """Minimise E_site(A) from A0 with L-BFGS (strong-Wolfe line search).  Returns the
    optimised raw tensor (CUDA float64) and the energy after every outer iteration."""
    A = torch.as_tensor(np.asarray(A0, dtype=np.float64) if not torch.is_tensor(A0) else A0,
                        dtype=torch.float64).cuda().clone().requires_grad_(True)
    hd = torch.as_tensor(h, dtype=torch.float64).cuda()
    opt = torch.optim.LBFGS([A], lr=lr, max_iter=1, history_size=history_size, line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        E = autograd.ctm_energy(A, chi, hd, warmup=warmup, k_tracked=k_tracked, precision=precision,
                                n_split=n_split)
        E.backward()
        return E

    energies = []
    for it in range(steps):
        E = opt.step(closure)
        energies.append(float(E.detach()))
        if callback is not None:
            callback(it, energies[-1], A)
    return A.detach(), energies
