"""Complex (E-irrep) QR-CTMRG oracle: plain numpy, complex128 (TEST INFRASTRUCTURE).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline import this module.  It restates App. A and Sec. II.B-C for
complex site tensors, step by step, with numpy einsum contractions and LAPACK's
QR (np.linalg.qr, with the gauge fixed here) and Hermitian eigenvalues as library
steps.  It shares no code with the CUDA path.

Symmetry (App. A).  The C3v group acts on A[s; i, j, k] (legs i, j, k carry the
x, y, z bonds) through
  * the three-fold rotation: U_C3 = (-1)^(d-1) e^{i phi} exp(i 2 pi/3 n.S) on the
    physical leg, n = (1,1,1)/sqrt(3), phi = 2 pi / 3, with a cyclic permutation of
    the virtual legs;
  * the reflection p_1 (normal m_1 = (1,-1,0)/sqrt(2)), anti-unitary:
    U_p = K C U_rot with U_rot = exp(i pi m_1.S) and K = i sigma_y for spin 1/2 (the
    matrix with +1, -1, ..., (-1)^(d+1) on the anti-diagonal), with the
    transposition of the x and y legs;
and the other elements follow by composition (the phases of U_p2, U_p3 are those
of r p_1 r^-1, r^2 p_1 r^-2).  Acting on a tensor, an anti-unitary element
conjugates the tensor and applies K conj(U_rot) to the physical leg.  The
projection averages A over the six elements.

Readings taken here (the paper's Fig. 2 and the sector drawings are not in the
text; each is pinned by tests/test_complex_oracle.py):
  * pairing: the rotation goes with the leg cycle T_r(A)[s; i, j, k] = U A[s; k, i, j]
    (the other direction breaks the equality of the x, y and z bond energies of the
    Kitaev-Heisenberg model that the C3 symmetry implies);
  * double layer a[(ii'),(jj'),(kk')] = sum_s A[s,i,j,k] conj(A[s,i',j',k']); the
    reflections then give a[l, u, z] = conj(a[u, l, z]) (and likewise for the other
    transpositions), with the fused ket-bra indices unchanged;
  * sector: the column edge is the complex conjugate of the row edge, so
      M[(a,y),(b,x)] = sum T[a,u,g] C[g,h] conj(T[b,l,h]) aB[u,l,z] aA[z,x,y]
    is Hermitian when C is; C' = sym(Q^H M Q)/|.| keeps C Hermitian, and the edge
    takes conj(Q) on its outer side and Q on its corner side:
      T'[i,x,j] = sum conj(Q[(a,y),i]) T[a,u,g] aB[u,w,z] aA[z,x,y] Q[(g,w),j];
  * reduced corner Y = M Q_prev S, S = diag(sgn C_ii) (C_ii real), and the QR gauge
    makes diag(R) real and >= 0;
  * bond types: the apex dimer's outer site B uses its legs in the order (x, y, z)
    with z radial, the inner site A the same tensor with z as its first leg
    (A[s; z, x, y] = A[s; x, y, z]), so the apex bond is a z bond for both ends and
    E_site = (3/2) Re tr(rho h_z) (C3 symmetry makes the x, y, z bonds equal);
  * for the real A1 representation (U_g = I, no conjugation) every step reduces to
    the real oracle;
  * transfer matrix (f2): the real path's column (edge, radial dimer, opposite edge,
    one Bravais vector along the edge) with the opposite edge conj(T), the mirror
    image of T as for the enlarged corner's column edge; then the spectrum is closed
    under complex conjugation (the reflections' anti-unitarity).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import oracle as real_oracle

__all__ = ["group_elements", "apply", "project", "double_layer", "open_layer", "enlarged_corner",
           "edge_update", "qr_gauge", "ComplexCTM", "spin_ops"]


def spin_ops(d: int = 2):
    S = (d - 1) / 2.0
    m = S - np.arange(d)
    Sz = np.diag(m).astype(np.complex128)
    Sp = np.zeros((d, d), dtype=np.complex128)
    for k in range(1, d):
        Sp[k - 1, k] = math.sqrt(S * (S + 1) - m[k] * (m[k] + 1))
    return (Sp + Sp.conj().T) / 2.0, (Sp - Sp.conj().T) / 2.0j, Sz


def _expm_herm(Hm, t):
    """exp(i t Hm) for a Hermitian matrix Hm (eigen-decomposition)."""
    w, V = np.linalg.eigh(Hm)
    return (V * np.exp(1j * t * w)[None, :]) @ V.conj().T


def _k_hat(d):
    K = np.zeros((d, d))
    for r in range(d):
        K[r, d - 1 - r] = (-1.0) ** r
    return K.astype(np.complex128)


def _generators(d, irrep):
    """(matrix, leg permutation, anti) of the rotation and of the reflection p_1."""
    if irrep == "A1":
        return (np.eye(d, dtype=np.complex128), (2, 0, 1), False), (np.eye(d, dtype=np.complex128), (1, 0, 2), False)
    Sx, Sy, Sz = spin_ops(d)
    n = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    m1 = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    nS = n[0] * Sx + n[1] * Sy + n[2] * Sz
    mS = m1[0] * Sx + m1[1] * Sy + m1[2] * Sz
    U_c3 = (-1.0) ** (d - 1) * np.exp(1j * 2.0 * math.pi / 3.0) * _expm_herm(nS, 2.0 * math.pi / 3.0)
    U_rot = _expm_herm(mS, math.pi)
    M_p = _k_hat(d) @ U_rot.conj()      # K C U_rot acting on conj(v)
    return (U_c3, (1, 2, 0), False), (M_p, (1, 0, 2), True)


def apply(el, A):
    """T_g(A)[s; i, j, k] = sum_t U[s,t] A'[t; legs permuted], A' = conj(A) if anti."""
    U, perm, anti = el
    B = A.conj() if anti else A
    B = np.transpose(B, (0, 1 + perm[0], 1 + perm[1], 1 + perm[2]))
    return np.einsum("st,tijk->sijk", U, B)


def _compose(g, h):
    """The element g after h: T_g(T_h(A))."""
    Ug, pg, ag = g
    Uh, ph, ah = h
    U = Ug @ (Uh.conj() if ag else Uh)
    perm = tuple(ph[pg[q]] for q in range(3))
    return (U, perm, ag != ah)


def group_elements(d: int = 2, irrep: str = "E"):
    """The six elements generated by the rotation and the reflection p_1 (closure by
    composition; an error if the generated set is not a group of order 6)."""
    r, p = _generators(d, irrep)
    e = (np.eye(d, dtype=np.complex128), (0, 1, 2), False)
    elems = [e]

    def same(x, y):
        return x[1] == y[1] and x[2] == y[2] and np.allclose(x[0], y[0], atol=1e-12)

    frontier = [r, p]
    while frontier:
        g = frontier.pop()
        if any(same(g, x) for x in elems):
            continue
        elems.append(g)
        for h in list(elems):
            frontier.append(_compose(g, h))
            frontier.append(_compose(h, g))
        if len(elems) > 6:
            raise ValueError("generators do not close into a group of order 6")
    if len(elems) != 6:
        raise ValueError("group of order %d" % len(elems))
    return elems


def project(A, irrep: str = "E", normalise: bool = True):
    """App. A: A_sym = (1/|G|) sum_g T_g(A), then unit Frobenius norm."""
    A = np.asarray(A, dtype=np.complex128)
    G = group_elements(A.shape[0], irrep)
    P = sum(apply(g, A) for g in G) / len(G)
    if normalise:
        P = P / np.linalg.norm(P)
    return P


def double_layer(K, B=None):
    """a[(ii'),(jj'),(kk')] = sum_s K[s,i,j,k] conj(B[s,i',j',k'])."""
    B = K if B is None else B
    D = K.shape[1]
    return np.einsum("sijk,slmn->iljmkn", K, B.conj()).reshape(D * D, D * D, D * D)


def open_layer(A, s, t, first_leg=0):
    """Open double layer A[s] (x) conj(A[t]) with the leg order rotated so that the
    leg `first_leg` of A comes first (0: x, y, z order)."""
    perm = [(first_leg + q) % 3 for q in range(3)]
    As = np.transpose(A[s], perm)
    At = np.transpose(A[t], perm)
    D = A.shape[1]
    return np.einsum("ijk,lmn->iljmkn", As, At.conj()).reshape(D * D, D * D, D * D)


def enlarged_corner(C, T, aB, aA):
    """Fig. 3c, one pair at a time: W = T C, X' = W conj(T), Y1 = X' aB, M = Y1 aA."""
    chi, D2 = T.shape[0], T.shape[1]
    W = np.einsum("aug,gh->auh", T, C, optimize=True)
    X = np.einsum("auh,blh->aulb", W, T.conj(), optimize=True)
    Y1 = np.einsum("aulb,ulz->abz", X, aB, optimize=True)
    return np.einsum("abz,zxy->aybx", Y1, aA, optimize=True).reshape(chi * D2, chi * D2)


def edge_update(T, aB, aA, Q):
    """T'[i,x,j] = sum conj(Q[(a,y),i]) T[a,u,g] aB[u,w,z] aA[z,x,y] Q[(g,w),j], unit norm,
    contracted one pair at a time."""
    chi, D2 = T.shape[0], T.shape[1]
    Q4 = Q.reshape(chi, D2, -1)
    H1 = np.einsum("aug,gwj->auwj", T, Q4, optimize=True)
    H2 = np.einsum("auwj,uwz->ajz", H1, aB, optimize=True)
    H3 = np.einsum("ajz,zxy->ajxy", H2, aA, optimize=True)
    Tn = np.einsum("ayi,ajxy->ixj", Q4.conj(), H3, optimize=True)
    return Tn / np.linalg.norm(Tn)


def qr_gauge(Y):
    """Thin QR (LAPACK) with diag(R) made real and >= 0 (column phases moved into Q)."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    dg = np.diag(R)
    ph = np.where(np.abs(dg) > 0.0, dg / np.where(np.abs(dg) > 0.0, np.abs(dg), 1.0), 1.0)
    return Q * ph[None, :], R * ph.conj()[:, None]


def corner_spectrum(C):
    w = np.abs(np.linalg.eigvalsh(0.5 * (C + C.conj().T)))
    w = np.sort(w)[::-1]
    return w / np.linalg.norm(w)


def transfer_apply(T, aB, aA, v):
    """f2 for complex environments (Sec. II.C, Fig. 4a): TM v for the column transfer
    matrix TM[(a,y,b),(g,w,h)] = sum T[a,u,g] aB[u,w,z] aA[z,x,y] conj(T[b,x,h]): one
    edge, one radial dimer and the opposite edge, advancing one Bravais vector along
    the edge (the real path's reading).  The opposite edge is the mirror image of T,
    conj(T), as the column edge of the enlarged corner is.  Contracted one pair at a
    time, v[g, w, h] in, out[a, y, b] out."""
    chi, D2 = T.shape[0], T.shape[1]
    V = np.asarray(v, dtype=np.complex128).reshape(chi, D2, chi)
    P1 = np.einsum("aug,gwh->auwh", T, V, optimize=True)
    P2 = np.einsum("auwh,uwz->ahz", P1, aB, optimize=True)
    P3 = np.einsum("ahz,zxy->axyh", P2, aA, optimize=True)
    return np.einsum("axyh,bxh->ayb", P3, T.conj(), optimize=True).reshape(-1)


def transfer_matrix(T, aB, aA):
    """The dense complex transfer matrix (chi D2 chi square; small cases)."""
    chi, D2 = T.shape[0], T.shape[1]
    N = chi * D2 * chi
    TM = np.einsum("aug,uwz,zxy,bxh->aybgwh", T, aB, aA, T.conj(), optimize=True)
    return TM.reshape(N, N)


def transfer_spectrum(T, aB, aA, nev: int = 3, dense_max: int = 4096):
    """The nev largest eigenvalue magnitudes of the transfer matrix normalised by the
    largest (lambda_i = |lambda_i'| / |lambda_0'|), xi = -1 / ln lambda_1 (Bravais
    steps) and the gap ln(lambda_1 / lambda_2) of the FCLS extrapolation (Eq. 3).
    LAPACK's general eigenvalues on the dense matrix when it is small, else ARPACK on
    transfer_apply."""
    chi, D2 = T.shape[0], T.shape[1]
    N = chi * D2 * chi
    if N <= dense_max:
        w = np.linalg.eigvals(transfer_matrix(T, aB, aA))
    else:
        import scipy.sparse.linalg as sla
        op = sla.LinearOperator((N, N), matvec=lambda v: transfer_apply(T, aB, aA, v), dtype=np.complex128)
        w = sla.eigs(op, k=max(nev, 3) + 2, which="LM", tol=1e-13, return_eigenvectors=False)
    lam = np.sort(np.abs(w))[::-1][:nev]
    lam = lam / lam[0]
    xi = -1.0 / np.log(lam[1]) if lam[1] > 0.0 else 0.0
    gap = np.log(lam[1] / lam[2]) if nev >= 3 and lam[2] > 0.0 else float("inf")
    return lam, xi, gap


class ComplexCTM:
    """QR-CTMRG of a complex C3v-symmetric tensor (irrep "E"; "A1" is the real case)."""

    def __init__(self, A, chi: int, irrep: str = "E", symmetrize: bool = True, projector: str = "qr",
                 corner: str = "qmq"):
        A = np.asarray(A, dtype=np.complex128)
        self.projector = projector      # "qr" (Sec. II.B) or "evd" (the conventional Fig. 3c projector)
        self.corner = corner            # "qmq" (Fig. 3a) or "r": the cheap variant from R
        self.A = project(A, irrep) if symmetrize else A / np.linalg.norm(A)
        self.irrep = irrep
        self.d, self.D = self.A.shape[0], self.A.shape[1]
        self.D2 = self.D * self.D
        self.chi = int(chi)
        self.n = self.chi * self.D2
        self.aB = double_layer(self.A)
        # site A: the same tensor with its z leg first (the apex bond is z at both ends)
        A_perm = np.transpose(self.A, (0, 3, 1, 2))
        self.aA = double_layer(A_perm)
        D, chi = self.D, self.chi
        diag = np.array([v * D + v for v in range(D)])
        t = self.aB[:, diag][:, :, diag].sum(axis=(1, 2))
        self.C = np.eye(chi, dtype=np.complex128)
        self.T = np.zeros((chi, self.D2, chi), dtype=np.complex128)
        for al in range(chi):
            self.T[al, :, al] = t
        self.Q = np.zeros((self.n, chi), dtype=np.complex128)
        self.Q[np.arange(chi), np.arange(chi)] = 1.0
        self.s = corner_spectrum(self.C)
        self.last = {}

    def set_env(self, C, T, Q):
        self.C, self.T, self.Q = (np.array(x, dtype=np.complex128) for x in (C, T, Q))
        self.s = corner_spectrum(self.C)

    def warm_start(self):
        S = np.where(np.real(np.diag(self.C)) < 0.0, -1.0, 1.0)
        return self.Q * S[None, :]

    def _projector(self, M):
        if self.projector == "evd":
            w, V = np.linalg.eigh(0.5 * (M + M.conj().T))
            keep = np.argsort(-np.abs(w), kind="stable")[: self.chi]
            return None, V[:, keep], None
        Y = M @ self.warm_start()
        Q, R = qr_gauge(Y)
        return Y, Q, R

    def step(self):
        M = enlarged_corner(self.C, self.T, self.aB, self.aA)
        S = np.where(np.real(np.diag(self.C)) < 0.0, -1.0, 1.0)
        Y, Q, R = self._projector(M)
        if self.corner == "r":
            # the cheap variant (Sec. II.B, Fig. 3d): R S = Q^H M Q_prev, which is Q^H M Q once
            # Q = Q_prev; S = diag(sgn C_jj) of the corner that entered the step
            Cr = R * S[None, :]
        else:
            Cr = Q.conj().T @ M @ Q
        Cn = 0.5 * (Cr + Cr.conj().T)
        Cn = Cn / np.linalg.norm(Cn)
        chi, D2 = self.chi, self.D2
        Tn = edge_update(self.T, self.aB, self.aA, Q)
        s = corner_spectrum(Cn)
        delta = float(np.linalg.norm(s - self.s))
        self.last = {"M": M, "Y": Y, "Q": Q, "R": R, "C": Cn, "T": Tn}
        self.C, self.T, self.Q, self.s = Cn, Tn, Q, s
        return delta

    def converge(self, max_steps: int, tol: float):
        delta = float("inf")
        for k in range(max_steps):
            delta = self.step()
            if delta < tol:
                return k + 1, delta
        return max_steps, delta

    def rho(self, bond_leg: int = 2):
        """Reduced density matrix of the apex bond; bond_leg selects which leg of the
        site tensor (0: x, 1: y, 2: z) plays the apex bond (the environment is the
        same for all three by the C3 symmetry of the double layer)."""
        d, chi = self.d, self.chi
        M = enlarged_corner(self.C, self.T, self.aB, self.aA)
        Q = self._projector(M)[1]
        Cr = Q.conj().T @ M @ Q
        Ch = 0.5 * (Cr + Cr.conj().T)
        Ch = Ch / np.linalg.norm(Ch)
        P5 = np.linalg.matrix_power(Ch, 5)
        # outer site B: legs rotated so bond_leg comes last; inner site A: bond_leg first
        fB, fA = (bond_leg + 1) % 3, bond_leg
        raw = np.zeros((d * d, d * d), dtype=np.complex128)
        for sA, sB, tA, tB in itertools.product(range(d), repeat=4):
            bB = open_layer(self.A, sB, tB, first_leg=fB)
            bA = open_layer(self.A, sA, tA, first_leg=fA)
            Moo = enlarged_corner(self.C, self.T, bB, bA)
            raw[sA * d + sB, tA * d + tB] = np.trace(P5 @ (Q.conj().T @ Moo @ Q))
        return raw / np.trace(raw)

    def transfer_spectrum(self, nev: int = 3):
        """f2: leading transfer-matrix eigenvalue magnitudes of the current environment, xi, gap."""
        return transfer_spectrum(self.T, self.aB, self.aA, nev)

    def energy(self, h):
        """(e_x, e_y, e_z, E_site): e_a = Re tr(rho_a h_a) on an a bond, E = (1/2) sum_a e_a."""
        e = []
        for a in range(3):
            r = self.rho(bond_leg=a)
            e.append(float(np.real(np.sum(r * np.asarray(h[a]).T))))
        return np.array(e), 0.5 * float(sum(e))
