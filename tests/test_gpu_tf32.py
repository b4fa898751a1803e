"""The TF32 tensor-core modes (CTM_SPLIT_TF32: A_hi B_hi + A_hi B_lo + A_lo B_hi; CTM_FP32_TF32:
A_hi B_hi alone) against FP64 products and the oracle.

Error model of one product C = A B with inner dimension K (elementwise, |A|, |B| taken
entrywise): the hi/lo slices represent each scaled operand to 2^-21 of its own magnitude
(the TF32 rounding of an FP32 value, 2^-22, plus that FP32 value's rounding, 2^-24), the
dropped A_lo B_lo term is below 2^-22 |a||b|, and FP32 accumulation of K terms adds at
most K 2^-23 of sum |a||b| (allowing truncating accumulation).  So
|C - C_hat| <= (3 2^-21 + K 2^-23) (|A| |B|).  With A_hi B_hi alone the operand term is
2 2^-11.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _gemm(A, B, prec):
    import torch
    from paper_2509_05090_gb300 import binding
    return _np(binding.ctm_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), prec, 2))


def _bound(A, B, prec):
    K = A.shape[1]
    op = 3 * 2.0 ** -21 if prec == "split_tf32" else 2 * 2.0 ** -11
    return (op + K * 2.0 ** -23) * (np.abs(A) @ np.abs(B))


@pytest.mark.parametrize("prec", ["split_tf32", "fp32_tf32"])
@pytest.mark.parametrize("M,N,K", [(300, 200, 150), (129, 65, 33), (72, 72, 2592), (2592, 72, 2592), (1, 1, 1)])
def test_tf32_gemm_within_bound(ctm_lib, prec, M, N, K):
    rng = np.random.default_rng(M + 7 * N + 13 * K)
    A = rng.uniform(-1, 1, (M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.uniform(-1, 1, (K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    C = _gemm(A, B, prec)
    ref = A @ B
    err = np.abs(C - ref)
    bound = _bound(A, B, prec)
    assert np.all(err <= bound), (err / bound).max()
    # and it is not vacuous: the split mode is far more accurate than one TF32 product
    if prec == "split_tf32" and K >= 150:
        assert (err / (np.abs(A) @ np.abs(B))).max() < 1e-5


def test_tf32_gemm_zero_and_scaled_rows(ctm_lib):
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (70, 40))
    A[5] = 0.0
    A[9] *= 1e-200
    A[11] *= 1e200
    B = rng.uniform(-1, 1, (40, 50))
    C = _gemm(A, B, "split_tf32")
    ref = A @ B
    assert np.all(C[5] == 0.0)
    assert np.all(np.abs(C - ref) <= _bound(A, B, "split_tf32"))


@pytest.mark.parametrize("prec", ["split_tf32", "fp32_tf32"])
def test_tf32_step_enlarged_corner_within_bound(ctm_lib, prec):
    """One step at D = 3, chi = 18 from the oracle's environment: the enlarged corner against
    the oracle within the chained bound (four products; each operand's error enters the next)."""
    from paper_2509_05090_gb300 import binding
    A = I.random_site_tensor(2, 3, 21)
    ref = O.OracleCTM(A, 18)
    for _ in range(3):
        ref.step()
    g = binding.CTM(A, 18, precision=prec)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    ref.step()
    g.ctm_step(1)
    M = _np(g.ctm_get_intermediate("M"))
    Mz = ref.last["M"]
    rel = np.abs(M - Mz).max() / np.abs(Mz).max()
    lim = 2e-5 if prec == "split_tf32" else 5e-2
    assert rel < lim, rel
    g.close()


@pytest.mark.parametrize("prec,tol", [("split_tf32", 2e-6), ("fp32_tf32", 2e-4)])
def test_tf32_converged_energy_against_oracle(ctm_lib, prec, tol):
    """heis_D2_chi8 converged in the TF32 modes.  Every contraction is accurate to the product
    bound above, (3 2^-21 + K 2^-23) relative with K <= n = 32 (5e-6) in the split mode and
    ~2^-10 with one product; the energy, a ratio of contractions of the converged
    environment, is held to 2e-6 and 2e-4 (measured on GB300: 2e-8 and 1.9e-5)."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["heis_D2_chi8"]
    A, h = w.site_tensor(), w.hamiltonians()
    ref = O.OracleCTM(A, w.chi)
    ref.converge(w.steps, w.tol)
    _, Ez = ref.energy(h)
    g = binding.CTM(A, w.chi, precision=prec)
    g.ctm_converge(max_steps=60, tol=1e-6 if prec == "split_tf32" else 1e-3)
    _, E, _ = g.ctm_energy(h)
    print(prec, "E", E, "oracle", Ez, "err", abs(E - Ez))
    assert abs(E - Ez) < tol, (E, Ez)
    g.close()
