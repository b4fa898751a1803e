"""Pins of the FP64 CPU oracle against facts the paper and mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
a textbook routine, a brute-force sum, an exactly solvable model or an
invariant the method must satisfy.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return float([ln for ln in f if ln.strip() and not ln.startswith("#")][0])


# ---------------------------------------------------------------- linear algebra

@pytest.mark.parametrize("n,k,rank", [(40, 8, 8), (64, 16, 5), (16, 16, 16), (33, 7, 7)])
def test_householder_qr_against_lapack(n, k, rank):
    rng = np.random.default_rng(n * 100 + k)
    Y = rng.standard_normal((n, rank)) @ rng.standard_normal((rank, k))
    Q, R = O.householder_qr(Y)
    assert np.allclose(Q.T @ Q, np.eye(k), atol=1e-13)
    assert np.all(np.abs(np.tril(R, -1)) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    assert np.linalg.norm(Y - Q @ R) <= 1e-13 * np.linalg.norm(Y)
    # textbook routine (LAPACK) with the same gauge, on the full-rank leading block
    Ql, Rl = np.linalg.qr(Y)
    sg = np.where(np.diag(Rl) < 0, -1.0, 1.0)
    Ql, Rl = Ql * sg, Rl * sg[:, None]
    lead = min(rank, k)
    assert np.allclose(R[:lead], Rl[:lead], atol=1e-11 * np.abs(R).max())
    assert np.allclose(Q[:, :lead], Ql[:, :lead], atol=1e-10)


def test_jacobi_eig_against_lapack():
    rng = np.random.default_rng(7)
    S = rng.standard_normal((24, 24))
    S = S + S.T
    w, V = O.sym_eig(S)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(S), atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(24), atol=1e-12)
    assert np.allclose(S @ V, V * w[None, :], atol=1e-11)


def test_corner_spectrum_is_normalised_singular_values():
    rng = np.random.default_rng(3)
    C = rng.standard_normal((12, 12))
    C = C + C.T
    s = O.corner_spectrum(C)
    sv = np.linalg.svd(C, compute_uv=False)
    assert np.allclose(s, sv / np.linalg.norm(sv), atol=1e-14)


# ---------------------------------------------------------------- a0, a1

def test_c3v_projection_is_s3_symmetric_and_idempotent():
    A = I.random_site_tensor(2, 3, 11)
    P = O.c3v_project(A)
    for perm in [(0, 2, 1, 3), (0, 1, 3, 2), (0, 3, 2, 1), (0, 2, 3, 1), (0, 3, 1, 2)]:
        assert np.allclose(P, P.transpose(perm), atol=1e-15)
    assert np.allclose(O.c3v_project(P), P, atol=1e-15)
    # the symmetric part is the orthogonal projection: residual orthogonal to it
    assert abs(np.sum((A - P) * P)) < 1e-12


def test_double_layer_against_einsum():
    A = I.random_site_tensor(3, 2, 5)
    a = O.double_layer(A)
    ref = np.einsum("sijk,slmn->iljmkn", A, A).reshape(4, 4, 4)
    assert np.allclose(a, ref, atol=1e-14)


# ---------------------------------------------------------------- a2, a6: brute force

def _random_env(chi, D2, seed, sym=True):
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((chi, chi))
    if sym:
        C = C + C.T
    T = rng.standard_normal((chi, D2, chi))
    return C, T


def test_enlarged_corner_brute_force():
    chi, D = 3, 2
    D2 = D * D
    A = O.prepare_site(I.random_site_tensor(2, D, 21))
    a = O.double_layer(A)
    rng = np.random.default_rng(2)
    aB = a + 0.1 * rng.standard_normal(a.shape)     # distinct tensors expose leg mix-ups
    aA = a + 0.1 * rng.standard_normal(a.shape)
    C, T = _random_env(chi, D2, 9, sym=False)
    M = O.enlarged_corner(C, T, aB, aA)
    ref = np.zeros((chi * D2, chi * D2))
    for al in range(chi):
        for y in range(D2):
            for be in range(chi):
                for x in range(D2):
                    s = 0.0
                    for u in range(D2):
                        for l in range(D2):
                            for z in range(D2):
                                tc = T[al, u, :] @ C @ T[be, l, :]
                                s += tc * aB[u, l, z] * aA[z, x, y]
                    ref[al * D2 + y, be * D2 + x] = s
    assert np.allclose(M, ref, atol=1e-12 * np.abs(ref).max())


def test_edge_update_brute_force():
    chi, D = 3, 2
    D2 = D * D
    rng = np.random.default_rng(4)
    aB = rng.standard_normal((D2, D2, D2))
    aA = rng.standard_normal((D2, D2, D2))
    _, T = _random_env(chi, D2, 10)
    Q, _ = np.linalg.qr(rng.standard_normal((chi * D2, chi)))
    Tn = O.edge_update(T, aB, aA, Q)
    ref = np.zeros((chi, D2, chi))
    for i in range(chi):
        for x in range(D2):
            for j in range(chi):
                s = 0.0
                for al in range(chi):
                    for y in range(D2):
                        for g in range(chi):
                            for w in range(D2):
                                q = Q[al * D2 + y, i] * Q[g * D2 + w, j]
                                if q == 0.0:
                                    continue
                                s += q * np.sum(T[al, :, g][:, None] * aB[:, w, :] * aA[:, x, y][None, :])
                ref[i, x, j] = s
    ref /= np.linalg.norm(ref)
    assert np.allclose(Tn, ref, atol=1e-12)


def test_enlarged_corner_symmetric_for_c3v_tensor():
    """Appendix A: the enlarged corner of a C3v-symmetric tensor is Hermitian."""
    A = O.prepare_site(I.random_site_tensor(2, 2, 31))
    a = O.double_layer(A)
    C, T = _random_env(5, 4, 12, sym=True)
    M = O.enlarged_corner(C, T, a, a)
    assert np.abs(M - M.T).max() <= 1e-14 * np.abs(M).max()


# ---------------------------------------------------------------- D = 1 product state

def test_product_state_exact():
    """D = 1: the environment is trivial and rho = (v v^T) (x) (v v^T) / |v|^4 exactly."""
    v = np.array([0.8, -0.35])
    A = I.product_site_tensor(v)
    ctm = O.OracleCTM(A, chi=4, symmetrize=False)
    ctm.converge(5, 1e-14)
    rho = ctm.rho()
    p = np.outer(v, v) / (v @ v)
    assert np.allclose(rho, np.kron(p, p), atol=1e-14)
    h = I.bond_hamiltonians(0.7, -0.4)
    e, E = O.bond_energies(rho, h)
    vv = v / np.linalg.norm(v)
    st = np.kron(vv, vv)
    exact = np.array([st @ h[a] @ st for a in range(3)])
    assert np.allclose(e, exact, atol=1e-14)
    assert abs(E - 0.5 * exact.sum()) < 1e-14


# ---------------------------------------------------------------- QR vs EVD projector

@pytest.mark.parametrize("chi", [8, 12])
def test_qr_ctmrg_matches_evd_ctmrg(chi):
    """Sec. III.B: QR- and EVD-based CTMRG reach the same energy and spectrum."""
    w = I.WORKLOADS["heis_D2_chi8"]
    h = I.bond_hamiltonians(0.0, 1.0)
    q = O.OracleCTM(w.site_tensor(), chi)
    steps, delta = q.converge(400, 1e-13)
    assert delta < 1e-13
    ev = O.OracleCTM(w.site_tensor(), chi, projector="evd")
    ev.set_env(q.C, q.T, q.Q)
    ev.converge(50, 1e-14)
    assert np.allclose(q.s, ev.s, atol=1e-10)
    assert abs(q.energy(h)[1] - ev.energy(h)[1]) < 1e-10


def test_converged_environment_invariants():
    """Fixed point: C diagonal up to slow basis rotation, rho a symmetric density matrix."""
    w = I.WORKLOADS["heis_D2_chi8"]
    q = O.OracleCTM(w.site_tensor(), w.chi)
    q.converge(300, 1e-13)
    assert np.abs(q.C - np.diag(np.diag(q.C))).max() < 1e-3
    rho = q.rho()
    assert abs(np.trace(rho) - 1.0) < 1e-14
    assert np.allclose(rho, rho.T, atol=1e-12)
    swap = np.zeros((4, 4))
    for s in range(2):
        for t in range(2):
            swap[s * 2 + t, t * 2 + s] = 1.0
    assert np.allclose(swap @ rho @ swap, rho, atol=1e-10)   # site A <-> site B
    assert np.linalg.eigvalsh(rho).min() > -1e-12


# ---------------------------------------------------------------- honeycomb Ising model

def _ising_exact_bond_correlation(beta, N=512):
    """<sigma_i sigma_j> on a bond of the infinite honeycomb Ising model.

    Exact free energy (Houtappel): -beta f = (3/4) ln 2 + (1/16 pi^2) int int
    ln[c^3 + 1 - s^2 (cos t1 + cos t2 + cos(t1 + t2))], c = cosh 2K, s = sinh 2K;
    there are 3/2 bonds per site, so <sigma sigma> = (2/3) d(-beta f)/dK.
    Midpoint rule, spectrally accurate away from the critical point.
    """
    t = (np.arange(N) + 0.5) * 2 * np.pi / N
    t1, t2 = np.meshgrid(t, t, indexing="ij")
    S = np.cos(t1) + np.cos(t2) + np.cos(t1 + t2)
    c, s = math.cosh(2 * beta), math.sinh(2 * beta)
    num = 6 * c * c * s - 4 * s * c * S
    den = c ** 3 + 1 - s * s * S
    return (2.0 / 3.0) * np.mean(num / den) / 4.0


def _ising_cylinder_bond_correlation(beta, L):
    """Brute-force transfer matrix on a brick-wall (honeycomb) cylinder of circumference L.

    Rows of L spins with periodic horizontal bonds; vertical bonds between rows
    r and r+1 only at columns c with (r + c) even.  Returns <sigma_c sigma_c+1>
    of a horizontal bond from the dominant left/right eigenvectors of the
    two-row transfer matrix.
    """
    sig = 1 - 2 * ((np.arange(2 ** L)[:, None] >> np.arange(L)[None, :]) & 1)   # (states, L)
    hor = np.sum(sig * np.roll(sig, -1, axis=1), axis=1)
    dh = np.exp(0.5 * beta * hor)              # D^{1/2}
    B = np.array([[math.exp(beta), math.exp(-beta)], [math.exp(-beta), math.exp(beta)]])
    J = np.ones((2, 2))

    def apply_V(psi, parity):
        t = psi.reshape((2,) * L)
        for c in range(L):
            mat = B if (c + parity) % 2 == 0 else J
            # state bit c of the flat index is the axis L-1-c of the reshaped array
            t = np.moveaxis(np.tensordot(mat, t, axes=([1], [L - 1 - c])), 0, L - 1 - c)
        return t.reshape(-1)

    def K(psi, parity):
        return dh * apply_V(dh * psi, parity)

    def dominant(first, second):
        psi = np.ones(2 ** L)
        for _ in range(400):
            new = K(K(psi, second), first)
            new /= np.linalg.norm(new)
            if np.linalg.norm(new - psi) < 1e-14:
                break
            psi = new
        return new

    right = dominant(0, 1)    # eigenvector of K0 K1
    left = dominant(1, 0)     # eigenvector of K1 K0 = (K0 K1)^T
    obs = sig[:, 0] * sig[:, 1]
    return float(np.sum(left * obs * right) / np.sum(left * right))


def test_ising_exact_formula_against_transfer_matrix():
    """Pins the exact-solution formula itself with brute force (independent of CTMRG)."""
    beta = 0.3
    ex = _ising_exact_bond_correlation(beta)
    errs = [abs(_ising_cylinder_bond_correlation(beta, L) - ex) for L in (10, 12, 14)]
    # finite-circumference error falls geometrically (about 10x per two columns)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6 and errs[1] / errs[2] > 5.0


@pytest.mark.parametrize("beta,chi,tol", [(0.3, 8, 1e-9), (0.5, 16, 1e-7)])
def test_ising_peps_pins_sector_wiring(beta, chi, tol):
    """<Psi|Psi> of the Ising tensor is the honeycomb Ising partition function, so
    4 <S^z S^z> from the CTMRG environment must equal the exact bond correlation.
    A mis-wired sector (wrong lattice) fails this."""
    A = I.ising_site_tensor(beta)
    ctm = O.OracleCTM(A, chi)
    steps, delta = ctm.converge(500, 1e-12)
    Sx, Sy, Sz = I.spin_matrices(2)
    hz = np.kron(Sz.real, Sz.real)
    e, _ = O.bond_energies(ctm.rho(), np.stack([hz, hz, hz]))
    assert abs(4 * e[2] - _ising_exact_bond_correlation(beta)) < tol


# ---------------------------------------------------------------- Kitaev point

def test_kitaev_exact_energy_golden_closed_form():
    """The paper's E_exact equals -(1/8) < |1 + e^{i q1} + e^{i q2}| > over the Brillouin zone."""
    golden = _read_golden("kitaev_exact_energy.txt")
    N = 2048
    q = (np.arange(N) + 0.5) * 2 * np.pi / N
    q1, q2 = np.meshgrid(q, q, indexing="ij")
    e = -np.mean(np.abs(1 + np.exp(1j * q1) + np.exp(1j * q2))) / 8.0
    assert abs(e - golden) < 5e-8


@pytest.mark.parametrize("seed,K", [(1000, -1.0), (1001, 1.0), (1002, -1.0)])
def test_kitaev_variational_bound(seed, K):
    """Sec. III.C: a variational energy never falls below the exact Kitaev energy."""
    golden = _read_golden("kitaev_exact_energy.txt")
    A = I.random_site_tensor(2, 2, seed)
    ctm = O.OracleCTM(A, 8)
    ctm.converge(200, 1e-11)
    _, E = ctm.energy(I.bond_hamiltonians(K, 0.0))
    assert E >= golden * abs(K) - 1e-12


def test_corner_from_r_identity_and_fixed_point():
    """Cheap corner variant C' = sym(R S)/|.|: the QR of Y = M Q_prev S gives
    R S = Q^T M Q_prev at any step (S^2 = I; a sign factor on the wrong side or a
    transposed R fails this), so it equals sym(Q^T M Q)/|.| once Q = Q_prev -- at the
    fixed point of the Ising PEPS (beta = 0.3, chi = 6), whose kept spectrum is well
    separated (at chi = 8 the cut falls inside a degenerate pair of M's eigenvalues)."""
    w = I.WORKLOADS["heis_D2_chi8"]
    ref = O.OracleCTM(w.site_tensor(), w.chi)
    for _ in range(3):
        ref.step()
    Qs = ref.warm_start()
    S = np.where(np.diag(ref.C) < 0.0, -1.0, 1.0)
    M = O.enlarged_corner(ref.C, ref.T, ref.a, ref.a)
    Q, R = O.householder_qr(O.matmul(M, Qs))
    assert np.max(np.abs(R * S[None, :] - Q.T @ M @ ref.Q)) <= 1e-13 * np.max(np.abs(R))
    early = np.max(np.abs(O.corner_from_r(R, ref.C) - O.corner_update(M, Q)))
    ising = O.OracleCTM(I.ising_site_tensor(0.3), 6)
    ising.converge(300, 1e-13)
    M = O.enlarged_corner(ising.C, ising.T, ising.a, ising.a)
    Q, R = O.householder_qr(O.matmul(M, ising.warm_start()))
    late = np.max(np.abs(O.corner_from_r(R, ising.C) - O.corner_update(M, Q)))
    assert late <= 1e-9 and early > 1e3 * late


def _zz3():
    Sz = np.diag([0.5, -0.5])
    hz = np.kron(Sz, Sz)
    return np.stack([hz, hz, hz])


def test_corner_from_r_iteration_reaches_the_same_fixed_point():
    """Iterating with the cheap corner variant converges to the environment of the
    standard QR-CTMRG when the kept spectrum has no near-degeneracy (Ising PEPS,
    beta = 0.3, chi = 6): the converged energies and corner spectra agree."""
    A = I.ising_site_tensor(0.3)
    a = O.OracleCTM(A, 6)
    b = O.OracleCTM(A, 6, corner="r")
    na, da = a.converge(400, 1e-13)
    nb, db = b.converge(400, 1e-13)
    assert da < 1e-13 and db < 1e-13
    assert abs(a.energy(_zz3())[1] - b.energy(_zz3())[1]) <= 1e-14
    assert np.max(np.abs(a.s - b.s)) <= 1e-10


def test_corner_from_r_is_inconsistent_while_the_basis_rotates():
    """The variant's limitation: on the random D = 2, chi = 8 state two kept eigenvalues
    of M are within 1 % of each other, so the orthogonal iteration turns the basis inside
    that pair by ~1e-2 per step long after the spectrum (delta < 1e-12) has converged.
    The standard corner Q^T M Q is covariant under that rotation; R S = Q^T M Q_prev is
    not, and the variant settles on a different energy."""
    w = I.WORKLOADS["heis_D2_chi8"]
    A, h = w.site_tensor(), w.hamiltonians()
    a = O.OracleCTM(A, w.chi)
    b = O.OracleCTM(A, w.chi, corner="r")
    a.converge(400, 1e-12)
    b.converge(400, 1e-12)
    Qp = a.Q.copy()
    a.step()
    assert np.max(np.abs(a.Q - Qp)) > 1e-3
    assert abs(a.energy(h)[1] - b.energy(h)[1]) > 1e-6


def test_pad_site_tensor_embeds_and_is_seeded():
    from paper_2509_05090_gb300.optimize import pad_site_tensor
    A = I.random_site_tensor(2, 3, 5)
    P1, P2 = pad_site_tensor(A, 5, 1e-2, 9), pad_site_tensor(A, 5, 1e-2, 9)
    assert P1.shape == (2, 5, 5, 5) and np.array_equal(P1, P2)
    assert np.array_equal(P1[:, :3, :3, :3], A)
    rest = P1.copy()
    rest[:, :3, :3, :3] = 0.0
    assert 0.0 < np.max(np.abs(rest)) <= 1e-2


def _ising_xi_along_chains(beta, L=12):
    """Correlation length of the honeycomb Ising model along a zigzag chain, in Bravais
    vectors: brute-force transfer matrix of a brick-wall cylinder (L rows, periodic)
    propagating along its chains, two columns (one Bravais vector) per step."""
    import scipy.sparse.linalg as sla
    sig = 1 - 2 * ((np.arange(2 ** L)[:, None] >> np.arange(L)[None, :]) & 1)

    def vert(par):
        e = np.zeros(2 ** L)
        for r in range(L):
            if (r + par) % 2 == 0:
                e += sig[:, r] * sig[:, (r + 1) % L]
        return np.exp(beta * e)

    v0, v1 = vert(0), vert(1)
    B = np.array([[math.exp(beta), math.exp(-beta)], [math.exp(-beta), math.exp(beta)]])

    def hor(psi):
        t = psi.reshape((2,) * L)
        for ax in range(L):
            t = np.moveaxis(np.tensordot(B, t, axes=([1], [ax])), 0, ax)
        return t.reshape(-1)

    op = sla.LinearOperator((2 ** L, 2 ** L), matvec=lambda p: v1 * hor(v0 * hor(p)), dtype=np.float64)
    w = np.sort(np.abs(sla.eigs(op, k=3, which="LM", return_eigenvectors=False)))[::-1]
    return -1.0 / np.log(w[1] / w[0])


def test_transfer_spectrum_pins_ising_correlation_length():
    """f2 (Sec. II.C, Eq. 3): the transfer matrix of the converged Ising-PEPS environment
    (beta = 0.3) gives xi(chi) rising toward the exact correlation length along the
    Bravais direction (brute-force cylinder transfer matrix), and the paper's
    extrapolation xi^-1(chi) = xi^-1(inf) + a ln(lambda_1/lambda_2) over chi = 16, 24
    lands on it.  A transfer matrix with the wrong column (another lattice direction or
    step) misses it by ~14 %."""
    beta = 0.3
    exact = _ising_xi_along_chains(beta)
    assert abs(exact - _ising_xi_along_chains(beta, 10)) < 1e-7        # converged in L
    res = []
    for chi in (8, 16, 24):
        ctm = O.OracleCTM(I.ising_site_tensor(beta), chi)
        ctm.converge(1000, 1e-13)
        lam, xi, gap = ctm.transfer_spectrum()
        res.append((xi, gap))
    assert res[0][0] < res[1][0] < res[2][0] < exact
    assert exact - res[2][0] < 0.005 * exact
    (x1, g1), (x2, g2) = res[1], res[2]
    slope = (1 / x1 - 1 / x2) / (g1 - g2)
    xi_inf = 1.0 / (1 / x2 - slope * g2)
    assert abs(xi_inf - exact) < 1e-4 * exact


def test_transfer_spectrum_product_state_and_apply():
    """D = 1 product state: with C = I, T = delta t the chi copies decouple and the
    transfer matrix is a multiple of the identity (every lambda_i = 1); and the
    matrix-free apply equals the dense matrix on a random vector."""
    ctm = O.OracleCTM(I.product_site_tensor([0.6, -0.8]), 4, symmetrize=False)
    ctm.converge(20, 1e-14)
    TM = O.transfer_matrix(ctm.T, ctm.a, ctm.a)
    assert np.max(np.abs(TM - TM[0, 0] * np.eye(TM.shape[0]))) <= 1e-14 * abs(TM[0, 0])
    w = I.WORKLOADS["heis_D2_chi8"]
    ref = O.OracleCTM(w.site_tensor(), w.chi)
    ref.step()
    v = np.random.default_rng(4).standard_normal(w.chi * w.D2 * w.chi)
    TM = O.transfer_matrix(ref.T, ref.a, ref.a)
    assert np.max(np.abs(TM @ v - O.transfer_apply(ref.T, ref.a, ref.a, v))) <= 1e-13 * np.max(np.abs(TM @ v))
