"""Parity of the complex (E-irrep) CUDA path with the complex oracle (App. A, Sec. II.B-C).

FP64: the contractions differ from the oracle only in rounding order, so the
enlarged corner agrees to a few ulps of its largest entry; Q and R are unique
(diag(R) real > 0), and a column j of Q can move by about n u (R_00 / R_jj), which
sets the per-column tolerance.  Split BF16 (T = 5 slices): every real product with
inner dimension K' has error below (T+1) 2^(-8T) K' max|a| max|b| per entry
(about 6e-12 K' relative), propagated the same way.
"""
import math

import numpy as np
import pytest

from oracle import complex_oracle as Z
from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -52


def _np(t):
    return t.detach().cpu().numpy()


def _kh(d, K, J):
    S = Z.spin_ops(d)
    heis = sum(np.kron(s, s) for s in S)
    return np.stack([K * np.kron(S[a], S[a]) + J * heis for a in range(3)])


def _ctm(A, chi, irrep="E", precision="fp64"):
    from paper_2509_05090_gb300 import binding
    return binding.CTMComplex(A, chi, irrep=irrep, precision=precision, n_split=5)


def _col_tol(R, n, scale):
    """First-order tolerance of each column of Q: scale * n u R_00 / R_jj."""
    dg = np.abs(np.diag(R))
    return scale * n * U64 * dg[0] / np.maximum(dg, 1e-300)


def _compare_step(g, z, label, mscale=64.0, qscale=64.0):
    """One step's outputs of the GPU context g against the oracle z (same inputs)."""
    M = _np(g.ctm_complex_get_intermediate("M"))
    Mz = z.last["M"]
    errM = np.abs(M - Mz).max() / np.abs(Mz).max()
    assert errM < mscale * U64 * math.sqrt(Mz.shape[0]), (label, "M", errM)
    R = _np(g.ctm_complex_get_intermediate("R"))
    Rz = z.last["R"]
    assert np.abs(np.diag(R).imag).max() < 1e-13 * abs(Rz[0, 0]), (label, "diag R imag")
    assert np.diag(R).real.min() >= 0.0
    Q = _np(g.ctm_complex_get_intermediate("Q"))
    Qz = z.last["Q"]
    tol = _col_tol(Rz, Qz.shape[0], qscale)
    errQ = np.abs(Q - Qz).max(axis=0)
    well = tol < 1e-4
    assert well.sum() >= 1
    assert np.all(errQ[well] < tol[well]), (label, "Q", errQ[well].max(), tol[well].min())
    return errM, errQ[well].max()


@pytest.mark.parametrize("d,D", [(2, 3), (3, 2)])
def test_complex_projection_and_double_layer(ctm_lib, d, D):
    A = I.random_complex_site_tensor(d, D, 41 + d)
    g = _ctm(A, chi=4)
    P = Z.project(A, "E")
    assert np.abs(_np(g.ctm_complex_get_intermediate("A")) - P).max() < 1e-14
    assert np.abs(_np(g.ctm_complex_get_intermediate("a")) - Z.double_layer(P)).max() < 1e-14
    g.close()


@pytest.mark.parametrize("D,chi,seed", [(2, 8, 51), (3, 12, 52), (2, 112, 53), (2, 160, 54), (2, 256, 55)])
def test_complex_steps_fp64(ctm_lib, D, chi, seed):
    """Random E-irrep tensors, ten steps in lockstep, each step from the oracle's environment
    (chi = 112: the embedded QR has 224 columns, beyond which U of its compact-WY solve no
    longer fits shared memory and is read from L2; chi = 160 and 256: the corner spectrum
    through the real 2chi x 2chi embedding on a thread-block cluster, and at 256 an embedded
    QR of 512 columns)."""
    A = I.random_complex_site_tensor(2, D, seed)
    g = _ctm(A, chi)
    z = Z.ComplexCTM(A, chi)
    for k in range(10):
        C, T, Q = z.C, z.T, z.Q
        if k > 0:
            g.ctm_complex_set_env(C, T, Q)
        dg = g.ctm_complex_step()
        dz = z.step()
        _compare_step(g, z, f"step {k}")
        Cg = _np(g.ctm_complex_get_intermediate("C"))
        assert np.abs(Cg - Cg.conj().T).max() == 0.0
        # C' and T' inherit the error of the well-determined part of Q
        assert np.abs(Cg - z.C).max() < 1e-9, (k, np.abs(Cg - z.C).max())
        assert abs(dg - dz) < 1e-9
        # the corner spectrum from the Hermitian tridiagonal reduction and bisection
        sg = _np(g.ctm_complex_get_intermediate("s"))
        assert np.abs(sg - z.s).max() < 1e-12, (k, np.abs(sg - z.s).max())


def test_complex_a1_matches_real_oracle(ctm_lib):
    A = I.random_site_tensor(2, 3, 61)
    g = _ctm(A.astype(np.complex128), 9, irrep="A1")
    r = O.OracleCTM(A, chi=9)
    for _ in range(6):
        g.ctm_complex_step()
        r.step()
    C = _np(g.ctm_complex_get_intermediate("C"))
    T = _np(g.ctm_complex_get_intermediate("T"))
    assert np.abs(C.imag).max() < 1e-14 and np.abs(T.imag).max() < 1e-14
    assert np.abs(C.real - r.C).max() < 1e-10
    assert np.abs(T.real - r.T).max() < 1e-10
    h = I.bond_hamiltonians(-0.6, 0.8)
    e, E, _ = g.ctm_complex_energy(h.astype(np.complex128))
    er, Er = r.energy(h)
    assert np.abs(e - er).max() < 1e-11 and abs(E - Er) < 1e-11


def test_complex_gauge_covariance_against_real_oracle(ctm_lib):
    """A real environment in a diagonal phase gauge stays that environment in that gauge."""
    rng = np.random.default_rng(71)
    D, chi = 2, 6
    A = I.random_site_tensor(2, D, 72)
    r = O.OracleCTM(A, chi=chi)
    for _ in range(4):
        r.step()
    W = np.exp(1j * rng.uniform(0, 2 * math.pi, chi))
    Wn = np.repeat(W, D * D)

    def gauge(C, T, Q):
        return (W.conj()[:, None] * C * W[None, :], W.conj()[:, None, None] * T * W[None, None, :],
                Wn.conj()[:, None] * Q * W[None, :])

    g = _ctm(A.astype(np.complex128), chi, irrep="A1")
    g.ctm_complex_set_env(*gauge(r.C, r.T, r.Q))
    for _ in range(4):
        r.step()
        g.ctm_complex_step()
        Cg, Tg, Qg = gauge(r.C, r.T, r.Q)
        C, T, Q = (_np(x) for x in g.ctm_complex_get_env())
        assert np.abs(C - Cg).max() < 1e-11
        assert np.abs(T - Tg).max() < 1e-11
        assert np.abs(Q - Qg).max() < 1e-10


@pytest.mark.parametrize("d,D,chi", [(2, 2, 8), (3, 2, 8)])
def test_complex_energy_fp64(ctm_lib, d, D, chi):
    v = I.coherent_state(d, (1.0, 1.0, 1.0) if d == 2 else (-1.0, -1.0, -1.0))
    A = I.complex_perturbed_product_site_tensor(v, D, 0.2, 81 + d)
    g = _ctm(A, chi)
    z = Z.ComplexCTM(A, chi)
    steps, delta, ok = g.ctm_complex_converge(60, 1e-10)
    z.converge(60, 1e-10)
    assert ok
    Cg = _np(g.ctm_complex_get_intermediate("C"))
    assert np.abs(np.sort(np.abs(np.linalg.eigvalsh(Cg)))[::-1] / np.linalg.norm(np.linalg.eigvalsh(Cg))
                  - z.s).max() < 1e-8
    for K, J in [(-1.0, 0.0), (-1.0, 0.4)]:
        h = _kh(d, K, J)
        e, E, rho = g.ctm_complex_energy(h)
        ez, Ez = z.energy(list(h))
        assert np.abs(e - ez).max() < 1e-9, (e, ez)
        assert abs(E - Ez) < 1e-9
        assert np.abs(e - e[2]).max() < 1e-9          # C3 covariance
        assert np.abs(rho - z.rho(bond_leg=2)).max() < 1e-9


def test_complex_split_steps_and_energy(ctm_lib):
    """Split BF16 (T = 5): step outputs against the oracle and the converged energy."""
    v = I.coherent_state(2, (1.0, 1.0, 1.0))
    A = I.complex_perturbed_product_site_tensor(v, 3, 0.05, 91)
    chi = 18
    g = _ctm(A, chi, precision="split_bf16")
    z = Z.ComplexCTM(A, chi)
    for k in range(3):
        if k > 0:
            g.ctm_complex_set_env(z.C, z.T, z.Q)
        g.ctm_complex_step()
        z.step()
        # split error of each real product: 6 * 2^-40 K' max|a| max|b| (K' <= 2 n); the
        # chained contractions of M add a few such terms
        n = z.n
        M = _np(g.ctm_complex_get_intermediate("M"))
        errM = np.abs(M - z.last["M"]).max() / np.abs(z.last["M"]).max()
        assert errM < 4 * 6 * 2.0 ** -40 * 2 * n, (k, errM)
    g.ctm_complex_set_env(z.C, z.T, z.Q)
    g.ctm_complex_converge(60, 1e-10)
    z.converge(60, 1e-10)
    h = _kh(2, -1.0, 0.3)
    e, E, _ = g.ctm_complex_energy(h)
    _, Ez = z.energy(list(h))
    assert abs(E - Ez) < 1e-9, (E, Ez)


@pytest.mark.parametrize("chi", [64, 72])
@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_complex_d6_workload(ctm_lib, precision, chi):
    """The D = 6 complex workloads (chi = 64, and 72 whose embedded QR has 144 columns):
    three steps of the random tensor against the oracle (M, and Q on its well-determined
    columns), then the converging tensor's energy."""
    w = I.WORKLOADS[f"kitaev_E_D6_chi{chi}"]
    A = w.site_tensor()
    g = _ctm(A, w.chi, precision=precision)
    z = Z.ComplexCTM(A, w.chi)
    scale = 64.0 if precision == "fp64" else 4 * 6 * 2.0 ** -40 / U64
    for k in range(3):
        if k > 0:
            g.ctm_complex_set_env(z.C, z.T, z.Q)
        g.ctm_complex_step()
        z.step()
        _compare_step(g, z, f"{precision} step {k}", mscale=scale * (1 if precision == "fp64" else 2 * math.sqrt(z.n)),
                      qscale=scale)
    g.close()
    w = I.WORKLOADS[f"kitaev_E_D6_chi{chi}_conv"]
    A = w.site_tensor()
    g = _ctm(A, w.chi, precision=precision)
    z = Z.ComplexCTM(A, w.chi)
    _, _, ok = g.ctm_complex_converge(40, 1e-10)
    assert ok
    z.converge(40, 1e-10)
    h = I.bond_hamiltonians(w.K, w.J, w.d).astype(np.complex128)
    e, E, _ = g.ctm_complex_energy(h)
    ez, Ez = z.energy(list(h))
    assert np.abs(e - ez).max() < 1e-9 and abs(E - Ez) < 1e-9, (e, ez)
    g.close()


def test_complex_rejects_bad_config(ctm_lib):
    from paper_2509_05090_gb300 import binding
    A = I.random_complex_site_tensor(2, 2, 3)
    with pytest.raises(binding.CtmError):
        binding.CTMComplex(A, 257)                      # chi above the embedded QR's 512 columns
    with pytest.raises(binding.CtmError):
        binding.CTMComplex(A[:1], 4)                    # d = 1 has no E irrep


def test_complex_graph_replay_equals_eager(ctm_lib):
    """Steps replayed from captured graphs (one-step and multi-step) follow the eager steps;
    the QR's FP64 atomics leave differences at rounding level only."""
    A = I.random_complex_site_tensor(2, 3, 101)
    g1, g2 = _ctm(A, 12), _ctm(A, 12)
    for _ in range(7):
        g1.ctm_complex_step(1)          # eager first, then the one-step graph
    g2.ctm_complex_step(1)
    g2.ctm_complex_step(6)              # one six-step graph
    for x, y in zip(g1.ctm_complex_get_env(), g2.ctm_complex_get_env()):
        assert np.abs(_np(x) - _np(y)).max() < 1e-11
    z = Z.ComplexCTM(A, 12)
    for _ in range(7):
        z.step()
    assert np.abs(_np(g1.ctm_complex_get_intermediate("C")) - z.C).max() < 1e-9


def test_complex_env_round_trip(ctm_lib):
    A = I.random_complex_site_tensor(2, 2, 102)
    g = _ctm(A, 8)
    g.ctm_complex_step(3)
    C, T, Q = g.ctm_complex_get_env()
    g.ctm_complex_set_env(C, T, Q)
    C2, T2, Q2 = g.ctm_complex_get_env()
    for x, y in ((C, C2), (T, T2), (Q, Q2)):
        assert np.array_equal(_np(x), _np(y))


def test_complex_unsymmetrised_tensor_follows_oracle(ctm_lib):
    """Without the projection M is not Hermitian; the step is the same formula on both sides."""
    from paper_2509_05090_gb300 import binding
    A = I.random_complex_site_tensor(2, 2, 103)
    g = binding.CTMComplex(A, 8, precision="fp64", symmetrize=False)
    z = Z.ComplexCTM(A, 8, symmetrize=False)
    assert np.abs(_np(g.ctm_complex_get_intermediate("A")) - z.A).max() < 1e-15
    for k in range(3):
        if k > 0:
            g.ctm_complex_set_env(z.C, z.T, z.Q)
        g.ctm_complex_step()
        z.step()
        M = _np(g.ctm_complex_get_intermediate("M"))
        assert np.abs(M - z.last["M"]).max() < 1e-13 * np.abs(z.last["M"]).max()
    g.close()


@pytest.mark.parametrize("prec,tol", [("split_tf32", 2e-6), ("fp32_tf32", 2e-4)])
def test_complex_tf32_energy(ctm_lib, prec, tol):
    """The TF32 engines under the complex path (their accuracy as in test_gpu_tf32.py)."""
    v = I.coherent_state(2, (1.0, 1.0, 1.0))
    A = I.complex_perturbed_product_site_tensor(v, 2, 0.2, 83)
    g = _ctm(A, 8, precision=prec)
    z = Z.ComplexCTM(A, 8)
    g.ctm_complex_converge(60, 1e-6 if prec == "split_tf32" else 1e-3)
    z.converge(60, 1e-10)
    h = _kh(2, -1.0, 0.3)
    _, E, _ = g.ctm_complex_energy(h)
    _, Ez = z.energy(list(h))
    print(prec, E, Ez, abs(E - Ez))
    assert abs(E - Ez) < tol, (E, Ez)
    g.close()


@pytest.mark.parametrize("precision,k", [("fp64", 1), ("split_bf16", 1), ("split_bf16", 3)])
def test_complex_pipelined_converge_matches_single_steps(ctm_lib, precision, k):
    """ctm_complex_converge's pipelined chunks (shifted corner spectra, deltas through
    pinned memory) against single-step calls: the step count the delta sequence
    implies, the last step's delta, and the same environment."""
    from test_gpu_paths import _pipelined_steps
    v = I.coherent_state(2, (1.0, 1.0, 1.0))
    A = I.complex_perturbed_product_site_tensor(v, 2, 0.2, 7)
    tol = 1e-10
    g1 = _ctm(A, 8, precision=precision)
    steps, delta, ok = g1.ctm_complex_converge(60, tol, k)
    assert ok and delta < tol
    g2 = _ctm(A, 8, precision=precision)
    deltas = [g2.ctm_complex_step(1) for _ in range(steps)]
    assert _pipelined_steps(deltas, k, tol, 60) == steps
    assert abs(delta - deltas[-1]) <= 1e-13 + 1e-6 * abs(deltas[-1])
    for x, y in zip(g1.ctm_complex_get_env(), g2.ctm_complex_get_env()):
        x, y = _np(x), _np(y)
        assert np.abs(x - y).max() <= 1e-10 * np.abs(y).max()
    g1.close()
    g2.close()


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_complex_deterministic_mode_bitwise_replays(ctm_lib, precision):
    """cfg.deterministic on the complex path (its embedded real QR sums per-CTA partials in a
    fixed order): eager single steps and a replayed multi-step graph give bit-identical
    environments."""
    from paper_2509_05090_gb300 import binding
    v = I.coherent_state(2, (1.0, 1.0, 1.0))
    A = I.complex_perturbed_product_site_tensor(v, 3, 0.2, 17)
    g1 = binding.CTMComplex(A, 18, irrep="E", precision=precision, n_split=5, deterministic=True)
    g2 = binding.CTMComplex(A, 18, irrep="E", precision=precision, n_split=5, deterministic=True)
    for _ in range(8):
        g1.ctm_complex_step(1)
    g2.ctm_complex_step(1)
    g2.ctm_complex_step(7)
    for x, y in zip(g1.ctm_complex_get_env(), g2.ctm_complex_get_env()):
        assert np.array_equal(_np(x), _np(y))
    g1.close()
    g2.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("split_bf16", 1e-8)])
def test_complex_transfer_spectrum_matches_oracle(ctm_lib, precision, tol):
    """f2 on the E irrep (Sec. II.C): the leading transfer-matrix magnitudes, xi and the
    FCLS gap of a converged complex environment against the complex oracle (dense
    eigenvalues), from the same environment."""
    A = I.random_complex_site_tensor(2, 2, 9)
    z = Z.ComplexCTM(A, 8)
    z.converge(80, 1e-11)
    lam_ref, xi_ref, gap_ref = z.transfer_spectrum(3)
    g = _ctm(A, 8, precision=precision)
    g.ctm_complex_set_env(z.C, z.T, z.Q)
    lam, xi, gap, iters, ok = g.ctm_complex_transfer_spectrum(nev=3, max_iter=2000, tol=1e-12)
    assert ok
    assert np.abs(lam - lam_ref).max() < tol
    assert abs(xi - xi_ref) < tol * 100 * max(1.0, xi_ref)
    assert abs(gap - gap_ref) < 1e-4 * max(1.0, abs(gap_ref))
    g.close()


def test_complex_transfer_spectrum_full_size(ctm_lib):
    """The complex transfer spectrum at D = 6, chi = 72 (vectors of 186624 complex entries) on
    the converging Kitaev workload, from the oracle's converged environment, against the
    oracle's ARPACK on its matrix-free transfer matrix.  On this near-product state the
    subleading magnitudes (~3e-6) lie in a cluster of nearly equal ones, which neither
    iteration resolves much below 1 % (the small-case test pins the operator to 1e-9);
    xi depends on lambda_1 only logarithmically."""
    w = I.WORKLOADS["kitaev_E_D6_chi72_conv"]
    A = w.site_tensor()
    z = Z.ComplexCTM(A, w.chi)
    z.converge(w.steps, w.tol)
    lam_ref, xi_ref, _ = z.transfer_spectrum(3)
    g = _ctm(A, w.chi, precision="split_bf16")
    g.ctm_complex_set_env(z.C, z.T, z.Q)
    # lambda_1, lambda_2 ~ 3e-6 sit in a cluster of near-equal magnitudes of this near-product
    # state, so the ratios are asked stable to 1e-9 between checks
    lam, xi, gap, iters, ok = g.ctm_complex_transfer_spectrum(nev=3, max_iter=400, tol=1e-9)
    assert ok, (lam, lam_ref, iters)
    assert abs(lam[0] - 1.0) < 1e-15
    assert np.abs(lam[1:] / lam_ref[1:] - 1.0).max() < 2e-2, (lam, lam_ref)
    assert abs(xi - xi_ref) < 1e-3 * xi_ref, (xi, xi_ref)
    g.close()


def test_complex_corner_from_r_matches_oracle(ctm_lib):
    """The cheap corner variant on the complex path (corner_mode 1): five FP64 steps, each
    from the oracle's environment, against the oracle's variant."""
    from paper_2509_05090_gb300 import binding
    A = I.random_complex_site_tensor(2, 2, 61)
    g = binding.CTMComplex(A, 8, irrep="E", precision="fp64", corner="r")
    z = Z.ComplexCTM(A, 8, corner="r")
    for k in range(5):
        if k > 0:
            g.ctm_complex_set_env(z.C, z.T, z.Q)
        dg = g.ctm_complex_step()
        dz = z.step()
        Cg = _np(g.ctm_complex_get_intermediate("C"))
        assert np.abs(Cg - z.C).max() < 1e-9, (k, np.abs(Cg - z.C).max())
        assert abs(dg - dz) < 1e-9
    g.close()
