"""Ragged batch (ctm_batch_*): every instance of a batch advanced in one graph
launch per step matches the FP64 oracle run on its own."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SMALL = [(2, 8, 31), (3, 9, 32), (2, 16, 33), (3, 24, 34), (1, 5, 35), (2, 13, 36)]   # (D, chi, seed)


@pytest.mark.parametrize("precision,tol_s,tol_e", [("fp64", 1e-10, 1e-12), ("split_bf16", 1e-8, 1e-9)])
def test_batch_instances_match_oracle(ctm_lib, precision, tol_s, tol_e):
    from paper_2509_05090_gb300 import binding
    tensors = [I.random_site_tensor(2, D, seed) for D, chi, seed in SMALL]
    chis = [chi for D, chi, seed in SMALL]
    batch = binding.CTMBatch(tensors, chis, precision=precision, n_split=5)
    steps = 6
    batch.ctm_batch_step(steps)
    h = I.bond_hamiltonians(0.4, 0.7)
    for i, (A, chi) in enumerate(zip(tensors, chis)):
        ref = O.OracleCTM(A, chi)
        for _ in range(steps):
            ref.step()
        g = batch.instance(i)
        s = g.ctm_get_intermediate("s").cpu().numpy()
        assert np.max(np.abs(s - ref.s)) <= tol_s, i
        _, E, _ = g.ctm_energy(h)
        assert abs(E - ref.energy(h)[1]) <= tol_e, i
    batch.close()


def test_batch96_runs_and_matches_standalone_instances(ctm_lib):
    """The 96-instance Kitaev-Heisenberg sweep (D in 3..6, chi in 24..72): all finite,
    and sampled instances equal the same instance advanced alone."""
    from paper_2509_05090_gb300 import binding
    wl = I.batch_workload()
    tensors = [w.site_tensor() for w in wl]
    batch = binding.CTMBatch(tensors, [w.chi for w in wl], precision="split_bf16", n_split=5)
    dmax = batch.ctm_batch_step(3, want_delta=True)
    assert np.isfinite(dmax)
    for i in (0, 17, 95):
        w = wl[i]
        alone = binding.CTM(tensors[i], w.chi, precision="split_bf16", n_split=5)
        alone.ctm_step(3)
        sb = batch.instance(i).ctm_get_intermediate("s").cpu().numpy()
        sa = alone.ctm_get_intermediate("s").cpu().numpy()
        assert np.max(np.abs(sb - sa)) <= 1e-9, i
        alone.close()
    batch.close()


def test_batch96_largest_instances_match_oracle(ctm_lib):
    """The 96-instance batch at its own sizes: after 3 batched steps, the three largest
    instances (n up to 2592) against the oracle run from the same initial environment
    (split-BF16 T = 5: spectrum 1e-8, energy 1e-9)."""
    from paper_2509_05090_gb300 import binding
    O.set_threads(0)
    wl = I.batch_workload()
    tensors = [w.site_tensor() for w in wl]
    batch = binding.CTMBatch(tensors, [w.chi for w in wl], precision="split_bf16", n_split=5)
    batch.ctm_batch_step(3)
    order = sorted(range(len(wl)), key=lambda i: -wl[i].n)[:3]
    for i in order:
        w = wl[i]
        ref = O.OracleCTM(tensors[i], w.chi)
        for _ in range(3):
            ref.step()
        g = batch.instance(i)
        s = g.ctm_get_intermediate("s").cpu().numpy()
        assert np.max(np.abs(s - ref.s)) <= 1e-8, i
        h = w.hamiltonians()
        e, E, rho = g.ctm_energy(h)
        assert abs(E - ref.energy(h)[1]) <= 1e-9, i
    batch.close()
