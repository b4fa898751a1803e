"""Pins of the complex (E-irrep) oracle against facts fixed outside it (App. A, Sec. II.B).

* the group: order 6, the rotation cubes to the identity, each reflection squares to
  it, the projection is idempotent (App. A);
* D = 1: the projection of any spin state is the state polarised along +n (spin 1/2)
  or the m = -1 state along n (spin 1), the only vectors the rotation fixes, and the
  product-state energy is the closed form K <S^a>^2 + J <S>.<S> per bond;
* the reflection Hermiticity of the double layer and the Hermiticity of the
  enlarged corner (Fig. 2b, Sec. II.A);
* a real A1 tensor reduces every step to the real C oracle;
* gauge covariance: a real environment rotated by a diagonal phase gauge must stay
  the same environment in that gauge through every step; a wrong placement of a
  complex conjugate in the corner or the edge update breaks this;
* C3 covariance of the bond energies of the Kitaev-Heisenberg model (e_x = e_y = e_z),
  which fixes the pairing of the rotation with the leg cycle;
* QR and EVD projectors reach the same fixed point;
* the column transfer matrix (f2): a real A1 tensor gives the real oracle's matrix,
  the matrix-free application equals the dense matrix, the spectrum is closed under
  complex conjugation with a real leading eigenvalue (which fixes the conjugated
  opposite edge; T on both sides breaks it), and a unitary change of the bond basis
  leaves the spectrum unchanged.
"""
import math

import numpy as np
import pytest

from oracle import complex_oracle as Z
from oracle import oracle as O


def _spin(d):
    return Z.spin_ops(d)


def _kh(d, K, J):
    S = _spin(d)
    heis = sum(np.kron(s, s) for s in S)
    return [K * np.kron(S[a], S[a]) + J * heis for a in range(3)]


def _n_state(d, m):
    """Eigenvector of n.S with eigenvalue m (n = (1,1,1)/sqrt 3)."""
    Sx, Sy, Sz = _spin(d)
    w, V = np.linalg.eigh((Sx + Sy + Sz) / math.sqrt(3.0))
    return V[:, int(np.argmin(np.abs(w - m)))]


def _near_product_E(D, eps, seed, d=2):
    rng = np.random.default_rng(seed)
    A = np.zeros((d, D, D, D), dtype=np.complex128)
    A[:, 0, 0, 0] = _n_state(d, 0.5 if d == 2 else -1.0)
    A += eps * (rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape))
    return A


@pytest.mark.parametrize("d", [2, 3])
def test_group_relations(d):
    G = Z.group_elements(d, "E")
    assert len(G) == 6
    r = next(g for g in G if g[1] == (1, 2, 0))
    U = r[0]
    assert np.abs(U @ U @ U - np.eye(d)).max() < 1e-13
    refl = [g for g in G if g[2]]
    assert len(refl) == 3
    for M, perm, _ in refl:
        assert sorted(perm) == [0, 1, 2] and sum(p != q for p, q in zip(perm, (0, 1, 2))) == 2
        assert np.abs(M @ M.conj() - np.eye(d)).max() < 1e-13        # the anti-unitary squares to 1
    rng = np.random.default_rng(3)
    A = rng.standard_normal((d, 2, 2, 2)) + 1j * rng.standard_normal((d, 2, 2, 2))
    P = Z.project(A, "E", normalise=False)
    assert np.abs(Z.project(P, "E", normalise=False) - P).max() < 1e-14
    for g in G:
        assert np.abs(Z.apply(g, P) - P).max() < 1e-14


@pytest.mark.parametrize("d,m", [(2, 0.5), (3, -1.0)])
def test_d1_projection_is_the_fixed_spin_state(d, m):
    rng = np.random.default_rng(5)
    v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    P = Z.project(v.reshape(d, 1, 1, 1), "E")[:, 0, 0, 0]
    ref = _n_state(d, m)
    assert abs(abs(np.vdot(ref, P)) - 1.0) < 1e-13


@pytest.mark.parametrize("d,m", [(2, 0.5), (3, -1.0)])
def test_product_state_energy(d, m):
    v = _n_state(d, m) * np.exp(0.7j)
    A = v.reshape(d, 1, 1, 1)
    ctm = Z.ComplexCTM(A, chi=1)
    ctm.converge(5, 1e-14)
    Sn = m / math.sqrt(3.0)                 # <S^a> = m n_a
    for K, J in [(-1.0, 0.0), (1.0, 0.5), (-0.6, -0.3)]:
        e, E = ctm.energy(_kh(d, K, J))
        e_ref = K * Sn * Sn + J * 3.0 * Sn * Sn
        assert np.abs(e - e_ref).max() < 1e-13
        assert abs(E - 1.5 * e_ref) < 1e-13


@pytest.mark.parametrize("D", [2, 3])
def test_reflection_hermiticity_and_hermitian_corner(D):
    rng = np.random.default_rng(11 + D)
    A = rng.standard_normal((2, D, D, D)) + 1j * rng.standard_normal((2, D, D, D))
    ctm = Z.ComplexCTM(A, chi=4 * D)
    a = ctm.aB
    for perm in [(1, 0, 2), (0, 2, 1), (2, 1, 0)]:
        assert np.abs(np.transpose(a, perm) - a.conj()).max() < 1e-14
    for perm in [(1, 2, 0), (2, 0, 1)]:
        assert np.abs(np.transpose(a, perm) - a).max() < 1e-14
    for _ in range(6):
        ctm.step()
        M = ctm.last["M"]
        assert np.abs(M - M.conj().T).max() < 1e-13 * np.abs(M).max()
        C = ctm.C
        assert np.abs(C - C.conj().T).max() < 1e-15
        Q = ctm.last["Q"]
        assert np.abs(Q.conj().T @ Q - np.eye(Q.shape[1])).max() < 1e-13
        assert np.abs(np.diag(ctm.last["R"]).imag).max() == 0.0
        assert np.diag(ctm.last["R"]).real.min() >= 0.0


def test_a1_reduces_to_real_oracle():
    rng = np.random.default_rng(21)
    A = rng.standard_normal((2, 3, 3, 3))
    real = O.OracleCTM(A, chi=9)
    cplx = Z.ComplexCTM(A.astype(np.complex128), chi=9, irrep="A1")
    assert np.abs(cplx.A - real.A).max() < 1e-15
    for _ in range(5):
        dr = real.step()
        dc = cplx.step()
        for key in ("M", "Y", "Q", "R", "C", "T"):
            x, y = real.last[key], cplx.last[key]
            assert np.abs(y.imag).max() < 1e-14
            assert np.abs(y.real - x).max() < 1e-12 * max(1.0, np.abs(x).max()), key
        assert abs(dr - dc) < 1e-12
    h = _kh(2, -1.0, 0.4)
    er, Er = real.energy(np.array([x.real for x in h]))
    ec, Ec = cplx.energy(h)
    assert np.abs(er - ec).max() < 1e-12 and abs(Er - Ec) < 1e-12


def test_gauge_covariance_fixes_conjugate_placement():
    rng = np.random.default_rng(31)
    D, chi = 2, 6
    A = rng.standard_normal((2, D, D, D))
    real = O.OracleCTM(A, chi=chi)
    for _ in range(4):
        real.step()
    D2, n = D * D, chi * D * D
    W = np.exp(1j * rng.uniform(0, 2 * math.pi, chi))
    Wn = np.repeat(W, D2)                  # W on the edge index of the (a, y) row multi-index

    def gauge(C, T, Q):
        Cg = W.conj()[:, None] * C * W[None, :]
        Tg = W.conj()[:, None, None] * T * W[None, None, :]
        Qg = Wn.conj()[:, None] * Q * W[None, :]
        return Cg, Tg, Qg

    cplx = Z.ComplexCTM(A.astype(np.complex128), chi=chi, irrep="A1")
    cplx.set_env(*gauge(real.C, real.T, real.Q))
    for _ in range(4):
        real.step()
        cplx.step()
        Cg, Tg, Qg = gauge(real.C, real.T, real.Q)
        assert np.abs(cplx.C - Cg).max() < 1e-12
        assert np.abs(cplx.T - Tg).max() < 1e-12
        assert np.abs(cplx.Q - Qg).max() < 1e-11
    h = _kh(2, -1.0, 0.4)
    er, _ = real.energy(np.array([x.real for x in h]))
    ec, _ = cplx.energy(h)
    assert np.abs(er - ec).max() < 1e-12


def test_gauge_covariance_detects_a_misplaced_conjugate():
    """The same check with the edge update's conjugate moved to the corner side."""
    rng = np.random.default_rng(31)
    D, chi = 2, 6
    A = rng.standard_normal((2, D, D, D))
    real = O.OracleCTM(A, chi=chi)
    for _ in range(4):
        real.step()
    W = np.exp(1j * rng.uniform(0, 2 * math.pi, chi))
    Wn = np.repeat(W, D * D)
    cplx = Z.ComplexCTM(A.astype(np.complex128), chi=chi, irrep="A1")
    cplx.set_env(W.conj()[:, None] * real.C * W[None, :], W.conj()[:, None, None] * real.T * W[None, None, :],
                 Wn.conj()[:, None] * real.Q * W[None, :])
    orig = Z.ComplexCTM.step

    def wrong_step(self):
        M = Z.enlarged_corner(self.C, self.T, self.aB, self.aA)
        Q, R = Z.qr_gauge(M @ self.warm_start())
        Cr = Q.conj().T @ M @ Q
        Cn = 0.5 * (Cr + Cr.conj().T)
        Cn /= np.linalg.norm(Cn)
        Tn = Z.edge_update(self.T, self.aB, self.aA, Q.conj())   # Q on the outer side, conj(Q) inside
        self.C, self.T, self.Q = Cn, Tn, Q
        return 0.0

    try:
        Z.ComplexCTM.step = wrong_step
        for _ in range(3):
            real.step()
            cplx.step()
    finally:
        Z.ComplexCTM.step = orig
    Cg = W.conj()[:, None] * real.C * W[None, :]
    assert np.abs(cplx.C - Cg).max() > 1e-6


def test_c3_covariance_of_bond_energies():
    A = _near_product_E(2, 0.3, 1)
    ctm = Z.ComplexCTM(A, chi=8)
    ctm.converge(80, 1e-10)
    for K, J in [(-1.0, 0.0), (-1.0, 0.3), (0.5, -1.0)]:
        e, E = ctm.energy(_kh(2, K, J))
        assert np.abs(e - e[2]).max() < 1e-10
        assert abs(E - 1.5 * e[2]) < 1e-10
    # the same energies from the z bond alone: rho_x, rho_y are rho_z rotated by U^2, U
    U = next(g for g in Z.group_elements(2, "E") if g[1] == (1, 2, 0))[0]
    rz = ctm.rho(bond_leg=2)
    rng = np.random.default_rng(2)
    h = [rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)) for _ in range(3)]
    h = [0.5 * (x + x.conj().T) for x in h]
    e, _ = ctm.energy(h)
    Wx, Wy = np.kron(U @ U, U @ U), np.kron(U, U)
    for a, Wa in [(0, Wx), (1, Wy), (2, np.eye(4))]:
        ea = np.real(np.sum((Wa @ rz @ Wa.conj().T) * h[a].T))
        assert abs(ea - e[a]) < 1e-10


def test_rho_is_a_density_matrix():
    A = _near_product_E(3, 0.2, 4)
    ctm = Z.ComplexCTM(A, chi=9)
    ctm.converge(60, 1e-9)
    r = ctm.rho()
    assert abs(np.trace(r) - 1.0) < 1e-13
    assert np.abs(r - r.conj().T).max() < 1e-8
    assert np.linalg.eigvalsh(0.5 * (r + r.conj().T)).min() > -1e-8


def test_qr_and_evd_reach_the_same_fixed_point():
    # chi = 6 cuts the corner spectrum in a gap (6.4e-4 kept, 5.5e-5 dropped), where the
    # QR iteration's subspace converges to the EVD's dominant eigenspace
    A = _near_product_E(2, 0.3, 1)
    qr = Z.ComplexCTM(A, chi=6)
    ev = Z.ComplexCTM(A, chi=6, projector="evd")
    # the EVD projector keeps the chi degenerate copies of the initial environment: it
    # starts from the QR iteration's environment after two steps instead
    qr.converge(2, 0.0)
    ev.set_env(qr.C, qr.T, qr.Q)
    qr.converge(150, 1e-10)
    ev.converge(150, 1e-10)
    assert np.abs(qr.s - ev.s).max() < 1e-10
    h = _kh(2, -1.0, 0.3)
    assert abs(qr.energy(h)[1] - ev.energy(h)[1]) < 1e-10


# ----------------------------------------------------------- transfer matrix (f2)
def _random_e_env(seed, D=2, chi=6, steps=60):
    from paper_2509_05090_gb300 import inputs as I
    z = Z.ComplexCTM(I.random_complex_site_tensor(2, D, seed), chi)
    z.converge(steps, 1e-11)
    return z


def test_transfer_a1_reduces_to_real_oracle():
    """A real A1 tensor: the complex transfer matrix is the real oracle's (pinned there by
    the exact Ising correlation length), entry by entry, with the same spectrum."""
    rng = np.random.default_rng(23)
    A = rng.standard_normal((2, 2, 2, 2))
    real = O.OracleCTM(A, chi=6)
    cplx = Z.ComplexCTM(A.astype(np.complex128), chi=6, irrep="A1")
    for _ in range(6):
        real.step()
        cplx.step()
    TMr = O.transfer_matrix(real.T, real.a, real.a)
    TMc = Z.transfer_matrix(cplx.T, cplx.aB, cplx.aA)
    assert np.abs(TMc.imag).max() < 1e-14
    assert np.abs(TMc.real - TMr).max() < 1e-12 * np.abs(TMr).max()
    lr, xr, gr = O.transfer_spectrum(real.T, real.a, real.a)
    lc, xc, gc = cplx.transfer_spectrum()
    assert np.abs(lr - lc).max() < 1e-10 and abs(xr - xc) < 1e-10


def test_transfer_apply_is_the_dense_matrix():
    z = _random_e_env(5)
    rng = np.random.default_rng(2)
    N = z.chi * z.D2 * z.chi
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    TM = Z.transfer_matrix(z.T, z.aB, z.aA)
    assert np.abs(Z.transfer_apply(z.T, z.aB, z.aA, v) - TM @ v).max() < 1e-13 * np.abs(TM).max() * N


@pytest.mark.parametrize("seed", [3, 9])
def test_transfer_spectrum_closed_under_conjugation(seed):
    """The reflections of the E-irrep state (anti-unitary) make the column transfer matrix
    equal to its complex conjugate in the basis with the two edges exchanged, so its
    spectrum is closed under conjugation and the leading eigenvalue is real.  That
    holds only with the opposite edge conjugated: the same column with T on both sides
    (a mistake planted here, in the oracle) loses it."""
    z = _random_e_env(seed)
    w = np.linalg.eigvals(Z.transfer_matrix(z.T, z.aB, z.aA))
    w = w[np.argsort(-np.abs(w))]
    scale = abs(w[0])
    assert max(np.min(np.abs(w - np.conj(x))) for x in w[:12]) < 1e-12 * scale
    assert abs(w[0].imag) < 1e-12 * scale and w[0].real > 0.0
    chi, D2 = z.chi, z.D2
    wrong = np.einsum("aug,uwz,zxy,bxh->aybgwh", z.T, z.aB, z.aA, z.T, optimize=True)
    ww = np.linalg.eigvals(wrong.reshape(chi * D2 * chi, -1))
    ww = ww[np.argsort(-np.abs(ww))]
    assert max(np.min(np.abs(ww - np.conj(x))) for x in ww[:12]) > 1e-6 * abs(ww[0])


def test_transfer_spectrum_gauge_invariant():
    """A unitary change of the environment's bond basis, T -> U T U^H (and C, Q with it),
    is a similarity of the transfer matrix: the same spectrum."""
    z = _random_e_env(4)
    rng = np.random.default_rng(12)
    X = rng.standard_normal((z.chi, z.chi)) + 1j * rng.standard_normal((z.chi, z.chi))
    U, _ = np.linalg.qr(X)
    T2 = np.einsum("ab,bug,hg->auh", U, z.T, U.conj(), optimize=True)
    l1, x1, g1 = Z.transfer_spectrum(z.T, z.aB, z.aA)
    l2, x2, g2 = Z.transfer_spectrum(T2, z.aB, z.aA)
    assert np.abs(l1 - l2).max() < 1e-12 and abs(x1 - x2) < 1e-10 and abs(g1 - g2) < 1e-8


# ----------------------------------------------------- cheap corner variant (f4)
def test_corner_from_r_identity_and_fixed_point():
    """C' = sym(R S)/|.| (S = diag(sgn Re C_jj)): R S = Q^H M Q_prev at every step (the QR of
    Y = M Q_prev S), and at a fixed point of the standard iteration whose Q is stationary
    one step of the variant gives the standard corner."""
    from paper_2509_05090_gb300 import inputs as I
    z = Z.ComplexCTM(I.random_complex_site_tensor(2, 2, 5), 8, corner="r")
    for _ in range(5):
        Qp, Cp = z.Q.copy(), z.C.copy()
        z.step()
        M, Q, R = z.last["M"], z.last["Q"], z.last["R"]
        S = np.where(np.real(np.diag(Cp)) < 0.0, -1.0, 1.0)
        assert np.abs(R * S[None, :] - Q.conj().T @ M @ Qp).max() < 1e-13 * np.abs(M).max()
    A = I.complex_perturbed_product_site_tensor(I.coherent_state(2, (1.0, 1.0, 1.0)), 2, 0.3, 7)
    zs = Z.ComplexCTM(A, 6)
    zs.converge(400, 1e-13)
    std = Z.ComplexCTM(A, 6)
    var = Z.ComplexCTM(A, 6, corner="r")
    for x in (std, var):
        x.set_env(zs.C, zs.T, zs.Q)
        x.step()
    assert np.abs(std.Q - zs.Q).max() < 1e-4          # Q stationary at this fixed point
    assert np.abs(var.C - std.C).max() < 1e-11
