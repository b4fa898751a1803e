"""GPU (libctm, FP64 path) against the FP64 CPU oracle, element by element.

Every call goes through the C ABI (paper_2509_05090_gb300.binding).  Step
parity feeds the oracle's own environment into one GPU step so rounding does
not compound; trajectory parity runs whole converging iterations.

Tolerances (FP64 throughout; both sides sum the same products in different
orders, so differences are a few ulps times the contraction length):
  * M, Y, A, a: max|diff| <= 1e-12 max|ref|
  * Q and R on the leading block of columns with R_ii / R_00 >= 1e-8 (beyond it Q
    is fixed only up to rounding): column j within max(1e-10 max|ref|, twice the
    first-order QR perturbation bound of the leading j + 1 columns for the measured
    Y difference plus the Householder backward error, split_bounds.qr_column_bounds)
    -- the leading block itself can be ill-conditioned (kappa ~ 1e7 on a
    converging near-product state);
  * C', T': whole, within 1e-10 max|ref|, when every column is leading; otherwise
    the block of columns whose Q bound is below 1e-10 max|Q|, each side scaled to
    unit norm on that block, plus Q_tail Q_tail^T Y within 1e-10 max|Y|;
  * spectra 1e-10, energies 1e-12 absolute.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _ctm(A, chi, **kw):
    from paper_2509_05090_gb300 import binding
    return binding.CTM(A, chi, **kw)


CASES = [
    ("heis_D2_chi8", 2, 2, 8, 1000),
    ("kitaev_D4_chi32", 2, 4, 32, 1001),
    ("ragged_D3_chi13", 2, 3, 13, 77),
    ("ragged_D2_chi70", 2, 2, 70, 78),
    ("spin1_D2_chi9", 3, 2, 9, 79),
]


@pytest.mark.parametrize("name,d,D,chi,seed", CASES)
def test_prepared_tensors_match_oracle(ctm_lib, name, d, D, chi, seed):
    A = I.random_site_tensor(d, D, seed)
    g = _ctm(A, chi)
    ref = O.OracleCTM(A, chi)
    assert _rel(_np(g.ctm_get_intermediate("A")), ref.A) <= 1e-14
    assert _rel(_np(g.ctm_get_intermediate("a")), ref.a) <= 1e-13
    C, T, Q = g.ctm_get_env()
    assert np.array_equal(_np(C), ref.C)
    assert _rel(_np(T), ref.T) <= 1e-13
    assert np.array_equal(_np(Q), ref.Q)
    g.close()


def _compare_last_step(g, ref, expect_full, T_in, tol_q=1e-10):
    """The GPU context's last step against the oracle's last step (ref.last and its
    environment); T_in is the edge that step started from.  expect_full: every column
    of R is leading (R_ii / R_00 >= 1e-8).  Returns the number of leading columns."""
    from split_bounds import edge_operator_fro, qr_column_bounds
    chi = ref.chi
    last = ref.last
    assert _rel(_np(g.ctm_get_intermediate("M")), last["M"]) <= 1e-12
    Y = _np(g.ctm_get_intermediate("Y"))
    assert _rel(Y, last["Y"]) <= 1e-12
    R_ref = last["R"]
    dR = np.abs(np.diag(R_ref))
    lead = int(np.sum(dR / dR[0] >= 1e-8))
    if expect_full is not None:
        assert (lead == chi) == expect_full, (lead, chi)
    R = _np(g.ctm_get_intermediate("R"))
    assert np.all(np.diag(R) >= 0.0)
    assert np.all(np.tril(R, -1) == 0.0)
    C, T, Q = (_np(x) for x in g.ctm_get_env())
    bq, br = qr_column_bounds(Y - last["Y"], last["Y"], R_ref, lead)
    qtol = np.maximum(tol_q * np.max(np.abs(last["Q"])), 2.0 * bq)
    rtol = np.maximum(tol_q * np.max(np.abs(R_ref)), 2.0 * br)
    assert np.all(np.max(np.abs(Q[:, :lead] - last["Q"][:, :lead]), axis=0) <= qtol)
    assert np.all(np.max(np.abs(R[:lead, :lead] - R_ref[:lead, :lead]), axis=0) <= rtol)
    assert np.max(np.abs(Q.T @ Q - np.eye(chi))) <= 1e-12
    if lead == chi:
        assert _rel(C, last["C"]) <= 1e-10
        assert _rel(T, last["T"]) <= 1e-10
    else:
        # tail rule: the part of Y outside the leading columns, from each side's own Q
        Pg = Q[:, lead:] @ (Q[:, lead:].T @ Y)
        Po = last["Q"][:, lead:] @ (last["Q"][:, lead:].T @ last["Y"])
        assert np.max(np.abs(Pg - Po)) <= 1e-10 * np.max(np.abs(last["Y"]))
        # C' and T' on the leading columns whose projector bound is below 1e-8 max|Q|,
        # each side scaled to unit norm on that block; tolerance: the first-order effect
        # of those columns' Q bound (2 ||M Q_w||_2 ||dQ_w||_F on the corner block,
        # 2 ||K||_F ||dQ_w||_F on the edge block), doubled for the scaling, floor 1e-10
        well = int(np.sum(np.cumsum(2.0 * bq > 1e-8 * np.max(np.abs(last["Q"]))) == 0))
        assert well >= 1
        Qw = last["Q"][:, :well]
        dQw = float(np.sqrt(np.sum((2.0 * bq[:well]) ** 2)))
        MQw = last["M"] @ Qw
        Cw = Qw.T @ MQw
        tol_c = max(1e-10, 4.0 * np.linalg.norm(MQw, 2) * dQw / np.linalg.norm(0.5 * (Cw + Cw.T)))
        D2 = ref.D2
        Qr = last["Q"].reshape(chi, D2, chi)
        Tw = np.einsum("ayi,ayxj->ixj", Qr[:, :, :well],
                       np.einsum("aug,uwz,zxy,gwj->ayxj", T_in, ref.a, ref.a, Qr[:, :, :well], optimize=True),
                       optimize=True)
        tol_t = max(1e-10, 4.0 * edge_operator_fro(T_in, ref.a) * dQw / np.linalg.norm(Tw))
        Cb, Cbr = C[:well, :well], last["C"][:well, :well]
        Tb, Tbr = T[:well, :, :well], last["T"][:well, :, :well]
        assert np.max(np.abs(Cb / np.linalg.norm(Cb) - Cbr / np.linalg.norm(Cbr))) <= tol_c
        assert np.max(np.abs(Tb / np.linalg.norm(Tb) - Tbr / np.linalg.norm(Tbr))) <= tol_t
        assert tol_c < 1e-4 and tol_t < 1e-4   # not vacuous
    assert np.max(np.abs(_np(g.ctm_get_intermediate("s")) - ref.s)) <= 1e-10
    return lead


def _step_parity(A, chi, pre_steps, expect_full=True, corner="qmq"):
    """One GPU step from the oracle's environment after pre_steps steps, compared with
    the oracle's step; the test asserts which comparison branch it took."""
    ref = O.OracleCTM(A, chi)
    for _ in range(pre_steps):
        ref.step()
    ref.corner = corner
    g = _ctm(A, chi, corner=corner)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    T_in = ref.T.copy()
    ref.step()
    g.ctm_step(1)
    lead = _compare_last_step(g, ref, expect_full, T_in)
    g.close()
    return lead


@pytest.mark.parametrize("name,d,D,chi,seed", CASES)
@pytest.mark.parametrize("pre", [0, 3])
def test_single_step_matches_oracle(ctm_lib, name, d, D, chi, seed, pre):
    A = I.random_site_tensor(d, D, seed)
    _step_parity(A, chi, pre)


def test_single_step_matches_oracle_d6_chi72(ctm_lib):
    """The benchmark workload (D = 6, chi = 72, enlarged corner 2592 x 2592), full size."""
    w = I.WORKLOADS["kh_D6_chi72"]
    _step_parity(w.site_tensor(), w.chi, 1)


def test_single_step_matches_oracle_chi144(ctm_lib):
    """chi = 144 (a QR of 144 columns) at D = 3 (n = 1296), from a non-trivial environment."""
    _step_parity(I.random_site_tensor(2, 3, 77), 144, 2)


@pytest.mark.parametrize("chi", [192, 224])
def test_single_step_matches_oracle_wide(ctm_lib, chi):
    """chi = 192 and 224 at D = 3: the QR's compact-WY solve reads U from L2 (more than 160
    columns); the corner spectrum runs on the thread-block cluster (chi >= 97)."""
    O.set_threads(0)
    _step_parity(I.random_site_tensor(2, 3, 78), chi, 2)


def test_single_step_matches_oracle_chi320(ctm_lib):
    """chi = 320 at D = 3 (n = 2880): the corner spectrum over the 16-CTA cluster (20 rows of
    C per CTA) and a QR of 320 columns.  Either comparison branch may apply."""
    O.set_threads(0)
    _step_parity(I.random_site_tensor(2, 3, 79), 320, 1, expect_full=None)


@pytest.mark.parametrize("D,chi,seed,pre", [(6, 72, None, 1), (3, 224, 78, 2), (2, 70, 78, 3)])
def test_single_step_matches_oracle_qr_slab(ctm_lib, monkeypatch, D, chi, seed, pre):
    """The QR with its row blocks in the global slab (the layout for shapes whose rows per
    SM do not fit shared memory, e.g. D = 6, chi = 512), forced by CTM_QR_SLAB=1 at sizes
    the oracle runs in seconds: the benchmark workload, 224 columns, and a ragged one
    (n = 280 over 140 CTAs of 2 rows)."""
    O.set_threads(0)
    monkeypatch.setenv("CTM_QR_SLAB", "1")
    A = I.WORKLOADS["kh_D6_chi72"].site_tensor() if seed is None else I.random_site_tensor(2, D, seed)
    _step_parity(A, chi, pre)


@pytest.mark.parametrize("name,pre", [("kh_D6_chi72_conv", 1), ("kitaev_D4_chi32_conv", 3)])
def test_single_step_matches_oracle_rank_deficient(ctm_lib, name, pre):
    """Converging near-product states: R falls below 1e-8 R_00 after ~16 / 37 columns, so
    the comparison takes the tail rule (leading block, Q_tail Q_tail^T Y, spectra)."""
    w = I.WORKLOADS[name]
    lead = _step_parity(w.site_tensor(), w.chi, pre, expect_full=False)
    assert lead < w.chi


def test_single_step_matches_oracle_d8_chi128(ctm_lib):
    """D = 8, chi = 128 (enlarged corner 8192 x 8192) from a non-trivial environment (the
    oracle after one step): M, Y, Q, R, C', T' and the spectrum element by element."""
    O.set_threads(0)
    w = I.WORKLOADS["kh_D8_chi128"]
    _step_parity(w.site_tensor(), w.chi, 1)


def test_trajectory_and_energy_match_oracle(ctm_lib):
    w = I.WORKLOADS["heis_D2_chi8"]
    A, h = w.site_tensor(), w.hamiltonians()
    ref = O.OracleCTM(A, w.chi)
    g = _ctm(A, w.chi)
    for k in range(w.steps):
        dr = ref.step()
        dg = g.ctm_step(1)
        assert abs(dg - dr) <= 1e-10 + 1e-8 * abs(dr)
    e_ref, E_ref = ref.energy(h)
    e, E, rho = g.ctm_energy(h)
    assert abs(E - E_ref) <= 1e-12
    assert np.max(np.abs(e - e_ref)) <= 1e-12
    assert np.max(np.abs(rho - ref.rho())) <= 1e-12
    g.close()


def test_trajectory_200_steps_converging_d4_chi32(ctm_lib):
    """200 steps from the initial environment on both sides (D = 4, chi = 32, converging
    near-product state; the iteration is contractive, so rounding differences stay at
    rounding level): delta of every step, the last step's M, Y, Q, R, C', T' and
    spectrum (tail rule), and the bond energies."""
    w = I.WORKLOADS["kitaev_D4_chi32_conv"]
    A, h = w.site_tensor(), w.hamiltonians()
    ref = O.OracleCTM(A, w.chi)
    g = _ctm(A, w.chi)
    for k in range(200):
        T_in = ref.T.copy()
        dr = ref.step()
        dg = g.ctm_step(1)
        assert abs(dg - dr) <= 1e-10 + 1e-8 * abs(dr), (k, dg, dr)
    _compare_last_step(g, ref, expect_full=False, T_in=T_in)
    e_ref, E_ref = ref.energy(h)
    e, E, rho = g.ctm_energy(h)
    assert abs(E - E_ref) <= 1e-12
    assert np.max(np.abs(e - e_ref)) <= 1e-12
    g.close()


def test_trajectory_random_d4_chi32_first_20_steps(ctm_lib):
    """The random D = 4, chi = 32 state: its iteration amplifies rounding differences by
    ~1e3 every 20 steps (test_trajectory_sensitivity; measured 1.6e-11 in M between GPU
    and oracle after 20 steps), so the environment itself is compared step by step
    elsewhere; here delta of each of 20 steps, the spectrum and the energies after them."""
    w = I.WORKLOADS["kitaev_D4_chi32"]
    A, h = w.site_tensor(), w.hamiltonians()
    ref = O.OracleCTM(A, w.chi)
    g = _ctm(A, w.chi)
    for k in range(20):
        dr = ref.step()
        dg = g.ctm_step(1)
        assert abs(dg - dr) <= 1e-10 + 1e-8 * abs(dr), (k, dg, dr)
    assert np.max(np.abs(_np(g.ctm_get_intermediate("s")) - ref.s)) <= 1e-10
    e_ref, E_ref = ref.energy(h)
    e, E, rho = g.ctm_energy(h)
    assert abs(E - E_ref) <= 1e-10
    g.close()


def test_energy_from_oracle_environment(ctm_lib):
    w = I.WORKLOADS["kitaev_D4_chi32"]
    A, h = w.site_tensor(), w.hamiltonians()
    ref = O.OracleCTM(A, w.chi)
    for _ in range(5):
        ref.step()
    g = _ctm(A, w.chi)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    e, E, rho = g.ctm_energy(h)
    e_ref, E_ref = ref.energy(h)
    assert abs(E - E_ref) <= 1e-12
    assert np.max(np.abs(e - e_ref)) <= 1e-12
    g.close()


def test_product_state_exact_on_gpu(ctm_lib):
    v = np.array([0.6, -0.8])
    g = _ctm(I.product_site_tensor(v), 5, symmetrize=False)
    g.ctm_converge(max_steps=10, tol=1e-14)
    h = I.bond_hamiltonians(0.3, 0.9)
    e, E, rho = g.ctm_energy(h)
    p = np.outer(v, v)
    assert np.max(np.abs(rho - np.kron(p, p))) <= 1e-14
    st = np.kron(v, v)
    assert np.allclose(e, [st @ h[a] @ st for a in range(3)], atol=1e-14)
    g.close()


def test_ising_bond_correlation_on_gpu(ctm_lib):
    from test_oracle_pins import _ising_exact_bond_correlation
    beta = 0.3
    g = _ctm(I.ising_site_tensor(beta), 8)
    steps, delta, ok = g.ctm_converge(max_steps=300, tol=1e-12)
    assert ok
    Sz = np.diag([0.5, -0.5])
    hz = np.kron(Sz, Sz)
    e, _, _ = g.ctm_energy(np.stack([hz, hz, hz]))
    assert abs(4 * e[2] - _ising_exact_bond_correlation(beta)) < 1e-9
    g.close()


def test_converge_graph_equals_eager_steps(ctm_lib):
    w = I.WORKLOADS["heis_D2_chi8"]
    A = w.site_tensor()
    g1 = _ctm(A, w.chi)
    g2 = _ctm(A, w.chi)
    steps, delta, ok = g1.ctm_converge(max_steps=20, tol=1e-300, check_every=5)
    assert steps == 20 and not ok
    g2.ctm_step(20)
    # the QR sums its partial dot products with FP64 atomics, so replays agree
    # to rounding, not bit for bit
    for x, y in zip(g1.ctm_get_env(), g2.ctm_get_env()):
        assert _rel(_np(x), _np(y)) <= 1e-12
    g1.close()
    g2.close()


def test_full_size_d8_chi128_first_step(ctm_lib):
    """D = 8, chi = 128 (enlarged corner 8192 x 8192): the first step from the
    initial environment, sampled M entries against the oracle's definition and
    the QR invariants on the full 8192 x 128 reduced corner."""
    w = I.WORKLOADS["kh_D8_chi128"]
    A = w.site_tensor()
    ref = O.OracleCTM(A, w.chi)          # oracle's own initial environment (cheap)
    g = _ctm(A, w.chi)
    g.ctm_step(1)
    M = _np(g.ctm_get_intermediate("M"))
    n, chi, D2 = w.n, w.chi, w.D2
    rng = np.random.default_rng(5)
    rows = rng.integers(0, n, 48)
    cols = rng.integers(0, n, 48)
    # block-diagonal start: M[(a,y),(b,x)] = delta_ab sum t_u t_l a[u,l,z] a[z,x,y]
    t = ref.T[0, :, 0]
    m = np.einsum("u,l,ulz,zxy->yx", t, t, ref.a, ref.a)
    for r, c in zip(rows, cols):
        exp = m[r % D2, c % D2] if (r // D2) == (c // D2) else 0.0
        assert abs(M[r, c] - exp) <= 1e-12 * np.max(np.abs(m))
    for b in range(0, chi, 37):   # whole diagonal blocks
        blk = M[b * D2:(b + 1) * D2, b * D2:(b + 1) * D2]
        assert _rel(blk, m) <= 1e-12
    Y = _np(g.ctm_get_intermediate("Y"))
    assert np.array_equal(Y, M[:, :chi])
    R = _np(g.ctm_get_intermediate("R"))
    C, T, Q = (_np(x) for x in g.ctm_get_env())
    assert np.max(np.abs(Q.T @ Q - np.eye(chi))) <= 1e-12
    assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
    assert np.linalg.norm(Y - Q @ R) <= 1e-13 * np.linalg.norm(Y)
    assert abs(np.linalg.norm(T) - 1) < 1e-13 and abs(np.linalg.norm(C) - 1) < 1e-13
    assert np.max(np.abs(C - C.T)) == 0.0
    g.close()


def test_nonfinite_input_rejected(ctm_lib):
    from paper_2509_05090_gb300 import binding
    A = I.random_site_tensor(2, 2, 3)
    A[1, 0, 1, 1] = np.nan
    with pytest.raises(binding.CtmError) as ei:
        _ctm(A, 8)
    assert ei.value.status == 5


def test_chi_one_and_d1(ctm_lib):
    A = I.random_site_tensor(2, 3, 12)
    _step_parity(A, 1, 2)
    _step_parity(I.random_site_tensor(2, 1, 4), 3, 1)


@pytest.mark.parametrize("name,pre", [("kitaev_D4_chi32", 3), ("kh_D6_chi72", 1)])
def test_corner_from_r_step_matches_oracle(ctm_lib, name, pre):
    """The cheap corner variant C' = sym(R S)/|.| (corner_mode 1), one FP64 step."""
    w = I.WORKLOADS[name]
    _step_parity(w.site_tensor(), w.chi, pre, corner="r")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("split_bf16", 1e-9)])
def test_corner_from_r_converged_energy_matches_oracle(ctm_lib, prec, tol):
    """The variant iterated for 30 steps on the Ising PEPS (beta = 0.3, chi = 6) in both
    precisions from the standard iteration's converged environment (the sign factor
    S = sgn C_jj is ill-defined while C has near-zero diagonal entries, as in the first
    steps from C = I, and R S is not invariant under it; at chi = 8 the cut falls inside
    a degenerate pair of M's eigenvalues, where rounding turns the kept basis): delta
    of every step and the bond energies against the oracle's variant."""
    A = I.ising_site_tensor(0.3)
    Sz = np.diag([0.5, -0.5])
    h = np.stack([np.kron(Sz, Sz)] * 3)
    start = O.OracleCTM(A, 6)
    start.converge(300, 1e-12)
    ref = O.OracleCTM(A, 6, corner="r")
    ref.set_env(start.C, start.T, start.Q)
    g = _ctm(A, 6, precision=prec, n_split=5, corner="r")
    g.ctm_set_env(start.C, start.T, start.Q)
    for k in range(30):
        dr = ref.step()
        dg = g.ctm_step(1)
        assert abs(dg - dr) <= 1e-10 + 1e-7 * abs(dr), (k, dg, dr)
    e_ref, E_ref = ref.energy(h)
    e, E, rho = g.ctm_energy(h)
    assert abs(E - E_ref) <= tol
    g.close()
