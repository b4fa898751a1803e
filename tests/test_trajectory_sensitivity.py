"""Why long trajectories of a random state are not compared element by element.

On the random Kitaev workload (D = 4, chi = 32) the corner spectrum has no gap at
chi, and the QR-CTMRG iteration carries a relative perturbation of 2e-16 of the site
tensor to O(1e-3) differences in the environment within 100 steps (the oracle
against itself).  No two correct implementations that round differently can agree
element by element over 200 such steps; the GPU trajectory tests therefore compare
the random state over 20 steps and a converging state over 200.
"""
import numpy as np

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I


def _run(A, chi, steps):
    ref = O.OracleCTM(A, chi)
    for _ in range(steps):
        ref.step()
    return ref


def test_random_state_trajectory_amplifies_rounding():
    O.set_threads(0)
    w = I.WORKLOADS["kitaev_D4_chi32"]
    A = w.site_tensor()
    A2 = A * (1.0 + 2e-16 * np.random.default_rng(3).standard_normal(A.shape))
    r20a, r20b = _run(A, w.chi, 20), _run(A2, w.chi, 20)
    d20 = np.max(np.abs(r20a.C - r20b.C)) / np.max(np.abs(r20a.C))
    for _ in range(80):
        r20a.step()
        r20b.step()
    d100 = np.max(np.abs(r20a.C - r20b.C)) / np.max(np.abs(r20a.C))
    assert d20 < 1e-11          # early steps: differences still near rounding
    assert d100 > 1e-6          # amplified by many orders of magnitude


def test_converging_state_trajectory_is_contractive():
    O.set_threads(0)
    w = I.WORKLOADS["kitaev_D4_chi32_conv"]
    A = w.site_tensor()
    A2 = A * (1.0 + 2e-16 * np.random.default_rng(3).standard_normal(A.shape))
    ra, rb = _run(A, w.chi, 100), _run(A2, w.chi, 100)
    assert np.max(np.abs(ra.s - rb.s)) < 1e-14
    Ca, Cb = ra.C[:16, :16], rb.C[:16, :16]
    assert np.max(np.abs(Ca / np.linalg.norm(Ca) - Cb / np.linalg.norm(Cb))) < 1e-13
