"""ctm_gemm_noalloc (library-owned fixed scratch, no device allocation) against ctm_gemm.

Collected last on purpose: it shares the library's static device scratch, and a
run that stops at the first failure has by then run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    (300, 130, 1000, "split_bf16", 5),   # split-K: integer accumulator in the scratch
    (257, 96, 64, "split_bf16", 3),
    (200, 72, 72, "fp64", 0),
    (64, 64, 2048, "fp64", 0),           # FP64 split-K partials in the scratch
]


def test_noalloc_gemm_matches_workspace_gemm_twice_in_a_row(ctm_lib):
    import torch
    from paper_2509_05090_gb300 import binding
    rng = np.random.default_rng(11)
    for call in range(2):
        for M, N, K, prec, T in CASES:
            A = torch.from_numpy(rng.standard_normal((M, K)))
            B = torch.from_numpy(rng.standard_normal((K, N)))
            ref = binding.ctm_gemm(A, B, prec, T if T else 4).cpu().numpy()
            got = binding.ctm_gemm_noalloc(A, B, prec, T if T else 4).cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (call, M, N, K, prec)


def test_noalloc_rejects_shapes_beyond_the_scratch(ctm_lib):
    import torch
    from paper_2509_05090_gb300 import binding
    A = torch.zeros((4096, 4096), dtype=torch.float64)
    B = torch.zeros((4096, 4096), dtype=torch.float64)
    with pytest.raises(binding.CtmError) as ei:
        binding.ctm_gemm_noalloc(A, B, "split_bf16", 5)
    assert ei.value.status == 2   # CTM_ENOMEM
