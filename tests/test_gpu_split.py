"""Split-BF16 tcgen05 contraction engine against the FP64 CPU oracle.

The engine evaluates C = A B as sum_{i+j<T} A_i B_j of BF16 digit slices with
exact per-chunk FP32 accumulation, so its error is the dropped-pair truncation:
|C_split - C|_{mn} <= (T + 1) 2^(-8T) K max_k|A_mk| max_k|B_kn| (the bound used
below, with the row/column maxima of the operands).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _split_gemm(A, B, T):
    import torch
    from paper_2509_05090_gb300 import binding
    return _np(binding.ctm_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), "split_bf16", T))


SHAPES = [(128, 64, 64), (200, 72, 72), (130, 100, 40), (64, 300, 520), (300, 130, 1000), (1024, 96, 4096),
          (96, 40, 5000),    # K > 4096: the two-launch transposed-operand pre-pass
          (64, 5000, 520),   # 5000 transposed rows: clusters beyond one wave, the two-launch pre-pass
          (40, 48, 12000)]   # K > 8192 (the enlarged corner's n at D = 5, chi = 480): the generic row pack


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("T", [2, 3, 4, 5])
def test_split_gemm_within_truncation_bound(ctm_lib, M, N, K, T):
    rng = np.random.default_rng(M * 7 + N * 3 + K + T)
    # rows and columns of very different scales exercise the per-row / per-column grids
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-20, 20, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp2(rng.integers(-20, 20, size=(1, N)))
    ref = O.matmul(A, B)
    C = _split_gemm(A, B, T)
    bound = (T + 1) * 2.0 ** (-8 * T) * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    assert np.all(np.abs(C - ref) <= bound)


def test_split_gemm_exact_on_small_integers(ctm_lib):
    """Integer operands that fit the top slice are multiplied exactly."""
    rng = np.random.default_rng(1)
    A = rng.integers(-128, 129, size=(256, 512)).astype(np.float64)
    B = rng.integers(-128, 129, size=(512, 96)).astype(np.float64)
    A[:, 0] = 128.0 * np.sign(A[:, 0] + 0.5)   # fixes the row grid at 2^8
    B[0, :] = 128.0
    # x 2^15 on that grid needs digits d_0, d_1 (d_2 = 0), so T = 3 keeps every
    # nonzero slice pair, including (1, 1)
    C = _split_gemm(A, B, 3)
    assert np.array_equal(C, A @ B)


def test_split_gemm_zero_rows_and_ragged(ctm_lib):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((77, 33))
    A[5] = 0.0
    B = rng.standard_normal((33, 19))
    B[:, 3] = 0.0
    C = _split_gemm(A, B, 5)
    ref = O.matmul(A, B)
    assert np.all(C[5] == 0.0) and np.all(C[:, 3] == 0.0)
    assert np.max(np.abs(C - ref)) <= 1e-10 * np.max(np.abs(ref))


def _ctm(A, chi, **kw):
    from paper_2509_05090_gb300 import binding
    return binding.CTM(A, chi, **kw)


@pytest.mark.parametrize("T,tol", [(3, 1e-4), (4, 1e-7), (5, 1e-9)])
def test_split_step_matches_oracle(ctm_lib, T, tol):
    w = I.WORKLOADS["kitaev_D4_chi32"]
    A = w.site_tensor()
    ref = O.OracleCTM(A, w.chi)
    for _ in range(3):
        ref.step()
    g = _ctm(A, w.chi, precision="split_bf16", n_split=T)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    ref.step()
    g.ctm_step(1)
    M = _np(g.ctm_get_intermediate("M"))
    assert np.max(np.abs(M - ref.last["M"])) <= tol * np.max(np.abs(ref.last["M"]))
    s = _np(g.ctm_get_intermediate("s"))
    assert np.max(np.abs(s - ref.s)) <= 100 * tol
    g.close()


def test_split_step_matches_oracle_d6_chi72(ctm_lib):
    """The benchmark workload (D = 6, chi = 72, n = 2592) in the benchmark's precision (T = 5),
    one step from the oracle's environment after one oracle step."""
    w = I.WORKLOADS["kh_D6_chi72"]
    A = w.site_tensor()
    ref = O.OracleCTM(A, w.chi)
    ref.step()
    g = _ctm(A, w.chi, precision="split_bf16", n_split=5)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    ref_Qs = ref.warm_start()
    ref.step()
    g.ctm_step(1)
    M = _np(g.ctm_get_intermediate("M"))
    assert np.max(np.abs(M - ref.last["M"])) <= 1e-9 * np.max(np.abs(ref.last["M"]))
    # Y = M Qs: the error of M carried through Qs plus this contraction's own truncation bound
    Qs = ref_Qs
    Mmax = np.max(np.abs(ref.last["M"]))
    bound = Mmax * (1e-9 * np.max(np.sum(np.abs(Qs), axis=0)) + 6 * 2.0 ** -40 * w.n * np.max(np.abs(Qs)))
    assert np.max(np.abs(_np(g.ctm_get_intermediate("Y")) - ref.last["Y"])) <= bound
    C, T, Q = (_np(x) for x in g.ctm_get_env())
    assert np.max(np.abs(Q.T @ Q - np.eye(w.chi))) <= 1e-12
    assert np.max(np.abs(_np(g.ctm_get_intermediate("s")) - ref.s)) <= 1e-7
    g.close()


def test_split_step_outputs_match_oracle_d6_chi72(ctm_lib):
    """M, Y, Q, R, C' and T' of one split-BF16 step (T = 5) at the benchmark size,
    element by element against the oracle's step from the same environment (the oracle
    after one step).  Tolerances (split_bounds): M and Y within the engine's truncation
    bound carried through their contraction chains; Q and R within the first-order QR
    perturbation bound of the measured Y difference plus the FP64 Householder backward
    error; C' and T' within their first-order bounds from the measured M difference,
    the Q bound and their own chains' truncation.  A factor 2 covers second-order
    terms.  The step has full column rank here (lead = chi)."""
    from split_bounds import corner_bound, edge_bound, enlarged_corner_err, gemm_err, qr_bounds
    w = I.WORKLOADS["kh_D6_chi72"]
    A = w.site_tensor()
    ref = O.OracleCTM(A, w.chi)
    ref.step()
    g = _ctm(A, w.chi, precision="split_bf16", n_split=5)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    C0, T0, Qs = ref.C.copy(), ref.T.copy(), ref.warm_start()
    ref.step()
    g.ctm_step(1)
    last = ref.last
    dRd = np.abs(np.diag(last["R"]))
    lead = int(np.sum(dRd / dRd[0] >= 1e-8))
    assert lead == w.chi
    eM = enlarged_corner_err(C0, T0, ref.a, 5)
    M = _np(g.ctm_get_intermediate("M"))
    assert np.all(np.abs(M - last["M"]) <= 2.0 * eM)
    eY = gemm_err(last["M"], Qs, 5, eA=eM)
    Y = _np(g.ctm_get_intermediate("Y"))
    assert np.all(np.abs(Y - last["Y"]) <= 2.0 * eY)
    dQ, dR = qr_bounds(float(np.linalg.norm(Y - last["Y"])), last["Y"], last["R"], lead)
    R = _np(g.ctm_get_intermediate("R"))
    assert np.all(np.diag(R) >= 0.0) and np.all(np.tril(R, -1) == 0.0)
    assert np.linalg.norm(R - last["R"]) <= 2.0 * dR
    C, T, Q = (_np(x) for x in g.ctm_get_env())
    assert np.linalg.norm(Q - last["Q"]) <= 2.0 * dQ
    dC = corner_bound(last["M"], last["Q"], float(np.linalg.norm(M - last["M"])), 2.0 * dQ, 5)
    assert np.linalg.norm(C - last["C"]) <= 2.0 * dC
    dT = edge_bound(T0, ref.a, last["Q"], 2.0 * dQ, 5)
    assert np.linalg.norm(T - last["T"]) <= 2.0 * dT
    # the bounds are not vacuous: far below the entries they bound (the truncation
    # terms are worst-case, K max|A| max|B|, so the C' and T' bounds are the loosest)
    for bound, x in ((2.0 * dQ, last["Q"]), (2.0 * dC, last["C"]), (2.0 * dT, last["T"])):
        assert bound < 1e-4 * np.max(np.abs(x))
    g.close()


@pytest.mark.parametrize("prec,tol", [("split_bf16", 1e-9), ("fp64", 1e-12)])
def test_energy_after_steps_matches_oracle_d6_chi72(ctm_lib, prec, tol):
    """Benchmark workload: three steps from the initial environment on each side, then
    the bond energies; split (T = 5) within 1e-9 of the FP64 oracle, FP64 within 1e-12."""
    w = I.WORKLOADS["kh_D6_chi72"]
    A, h = w.site_tensor(), w.hamiltonians()
    O.set_threads(0)
    ref = O.OracleCTM(A, w.chi)
    for _ in range(3):
        ref.step()
    e_ref, E_ref = ref.energy(h)
    g = _ctm(A, w.chi, precision=prec, n_split=5)
    g.ctm_step(3)
    e, E, rho = g.ctm_energy(h)
    assert abs(E - E_ref) <= tol
    assert np.max(np.abs(e - e_ref)) <= tol
    g.close()


@pytest.mark.parametrize("prec,tol", [("split_bf16", 1e-9), ("fp64", 1e-12)])
def test_converged_energy_matches_oracle_d6_chi72(ctm_lib, prec, tol):
    """Converging workload at the benchmark size (near-product state, D = 6, chi = 72):
    both sides iterate to delta < 1e-10, then the energies agree within 1e-9 (split) /
    1e-12 (FP64) -- the mixed-vs-FP64 energy criterion against the oracle itself."""
    w = I.WORKLOADS["kh_D6_chi72_conv"]
    A, h = w.site_tensor(), w.hamiltonians()
    O.set_threads(0)
    ref = O.OracleCTM(A, w.chi)
    rsteps, rdelta = ref.converge(w.steps, w.tol)
    assert rdelta < w.tol
    e_ref, E_ref = ref.energy(h)
    g = _ctm(A, w.chi, precision=prec, n_split=5)
    steps, delta, ok = g.ctm_converge(max_steps=w.steps, tol=w.tol, check_every=1)
    assert ok and abs(steps - rsteps) <= 2
    e, E, rho = g.ctm_energy(h)
    assert abs(E - E_ref) <= tol
    assert np.max(np.abs(e - e_ref)) <= tol
    g.close()


def test_split_energy_error_below_1e9(ctm_lib):
    """Mixed precision (T = 5 slices) reaches the FP64 oracle's converged energy within 1e-9."""
    w = I.WORKLOADS["heis_D2_chi8"]
    A, h = w.site_tensor(), w.hamiltonians()
    ref = O.OracleCTM(A, w.chi)
    ref.converge(300, 1e-12)
    _, E_ref = ref.energy(h)
    g = _ctm(A, w.chi, precision="split_bf16", n_split=5)
    steps, delta, ok = g.ctm_converge(max_steps=300, tol=1e-12)
    e, E, rho = g.ctm_energy(h)
    assert abs(E - E_ref) <= 1e-9
    g.close()


def test_split_step_outputs_match_oracle_d8_chi128(ctm_lib):
    """D = 8, chi = 128 (enlarged corner 8192 x 8192) in split-BF16 (T = 5), one step from
    the oracle's environment after one step: M and Y within the derived chain bounds,
    Q and R within the first-order QR bound of the measured Y difference, C' and T' within
    their first-order bounds (as at D = 6, split_bounds)."""
    from split_bounds import corner_bound, edge_bound, enlarged_corner_err, gemm_err, qr_bounds
    O.set_threads(0)
    w = I.WORKLOADS["kh_D8_chi128"]
    A = w.site_tensor()
    ref = O.OracleCTM(A, w.chi)
    ref.step()
    g = _ctm(A, w.chi, precision="split_bf16", n_split=5)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    C0, T0, Qs = ref.C.copy(), ref.T.copy(), ref.warm_start()
    ref.step()
    g.ctm_step(1)
    last = ref.last
    dRd = np.abs(np.diag(last["R"]))
    lead = int(np.sum(dRd / dRd[0] >= 1e-8))
    assert lead == w.chi
    eM = enlarged_corner_err(C0, T0, ref.a, 5)
    M = _np(g.ctm_get_intermediate("M"))
    assert np.all(np.abs(M - last["M"]) <= 2.0 * eM)
    eY = gemm_err(last["M"], Qs, 5, eA=eM)
    del eM
    Y = _np(g.ctm_get_intermediate("Y"))
    assert np.all(np.abs(Y - last["Y"]) <= 2.0 * eY)
    dQ, dR = qr_bounds(float(np.linalg.norm(Y - last["Y"])), last["Y"], last["R"], lead)
    R = _np(g.ctm_get_intermediate("R"))
    assert np.linalg.norm(R - last["R"]) <= 2.0 * dR
    C, T, Q = (_np(x) for x in g.ctm_get_env())
    assert np.linalg.norm(Q - last["Q"]) <= 2.0 * dQ
    dC = corner_bound(last["M"], last["Q"], float(np.linalg.norm(M - last["M"])), 2.0 * dQ, 5)
    assert np.linalg.norm(C - last["C"]) <= 2.0 * dC
    dT = edge_bound(T0, ref.a, last["Q"], 2.0 * dQ, 5)
    assert np.linalg.norm(T - last["T"]) <= 2.0 * dT
    # not vacuous; the worst-case truncation terms K max|A| max|B| grow with K (8192 here)
    for bound, x in ((2.0 * dQ, last["Q"]), (2.0 * dC, last["C"]), (2.0 * dT, last["T"])):
        assert bound < 1e-3 * np.max(np.abs(x))
    g.close()
