"""Large environments (chi > 224) at full size, through the C ABI.

Heisenberg D = 5, chi = 480 (n = 12000): one SM's share of the QR's rows (79 rows of
481 doubles) does not fit shared memory, so the row blocks live in the global slab,
and the corner spectrum runs over a 16-CTA thread-block cluster (30 rows of C per
CTA).  The oracle's step at this size takes minutes, so the checks are properties
that hold at any size
(Sec. II.B: Y = Q R with Q orthonormal and diag(R) >= 0; the corner spectrum is the
normalised |eigenvalues| of the symmetric corner), plus the split-BF16 step against
the library's FP64 step from the same environment.  The same kernels are compared
with the oracle element by element at chi = 320 and with the slab forced at small
sizes (test_gpu_parity.py).
"""
import numpy as np
import pytest

from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def test_large_chi_step_properties_and_split_vs_fp64(ctm_lib):
    import torch
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["heis_D5_chi480"]
    A, h = w.site_tensor(), w.hamiltonians()
    g = binding.CTM(A, w.chi, precision="split_bf16", n_split=5)
    for _ in range(2):
        d = g.ctm_step(1)
        assert np.isfinite(d) and d > 0.0
    # Y = Q R, Q^T Q = I, R upper triangular with a non-negative diagonal
    Y = g.ctm_get_intermediate("Y")
    R = g.ctm_get_intermediate("R")
    Q = g.ctm_get_intermediate("Q")
    eye = torch.eye(w.chi, dtype=torch.float64, device="cuda")
    assert float((Q.T @ Q - eye).abs().max()) <= 1e-12
    assert bool((torch.diagonal(R) >= 0).all())
    assert bool((torch.tril(R, -1) == 0).all())
    assert float((Y - Q @ R).abs().max()) <= 1e-12 * float(Y.abs().max())
    # the corner spectrum against a dense symmetric eigensolver on the same corner
    C, T, Qe = g.ctm_get_env()
    Cn = _np(C)
    assert np.max(np.abs(Cn - Cn.T)) == 0.0
    lam = np.sort(np.abs(np.linalg.eigvalsh(Cn)))[::-1]
    s_ref = lam / np.linalg.norm(lam)
    s = _np(g.ctm_get_intermediate("s"))
    assert np.max(np.abs(s - s_ref)) <= 1e-12
    # one more step in split BF16 and in FP64 from the same environment: energies agree
    # within the mixed-precision bound the benchmark states (1e-9)
    f = binding.CTM(A, w.chi, precision="fp64")
    f.ctm_set_env(C, T, Qe)
    g.ctm_step(1)
    f.ctm_step(1)
    _, Eg, _ = g.ctm_energy(h)
    _, Ef, _ = f.ctm_energy(h)
    assert np.isfinite(Ef) and abs(Eg - Ef) <= 1e-9, (Eg, Ef)
    sg = _np(g.ctm_get_intermediate("s"))
    sf = _np(f.ctm_get_intermediate("s"))
    assert np.max(np.abs(sg - sf)) <= 1e-8
    g.close()
    f.close()


def test_large_chi_converge_pipelined(ctm_lib):
    """ctm_converge at chi = 360 (the cluster spectrum, ~5 ms, runs on the side stream across
    the pipelined graphs): the deltas it reports match those of single steps from the same
    start."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["heis_D5_chi360"]
    A = w.site_tensor()
    a = binding.CTM(A, w.chi, precision="fp64")
    ds = [a.ctm_step(1) for _ in range(4)]
    b = binding.CTM(A, w.chi, precision="fp64")
    steps, delta, ok = b.ctm_converge(max_steps=4, tol=1e-300, check_every=1)
    assert steps == 4 and not ok
    assert abs(delta - ds[-1]) <= 1e-12 * max(1.0, abs(ds[-1]))
    a.close()
    b.close()
