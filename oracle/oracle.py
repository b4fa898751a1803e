"""Python driver of the FP64 CPU oracle (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The arithmetic lives in ``ctm_oracle.c``
(plain loops, FP64); this file marshals numpy arrays and strings the steps of
one QR-based CTMRG iteration together in the paper's order (Sec. II.B, Fig. 3):

    enlarged corner M  ->  reduced corner Y = M Q_prev  ->  Householder QR
    (gauge diag R >= 0)  ->  C' = sym(Q^T M Q) / norm  ->  T' = Q^T (T a a) Q / norm
    ->  corner spectrum and its change delta.

Readings of the paper taken here (the drawings of Fig. 1 and Fig. 3 are not in
the text):
  * reduced corner: Y = M Q_prev S with S = diag(sgn C_ii) (sgn 0 = +1), one
    orthogonal-iteration step warm-started from the previous projector;
    Q_0 = first chi columns of the identity.  At a fixed point C is diagonal
    (C = Q^T M Q with M Q = Q R), so S makes Y = Q |Lambda| and the positive
    diag(R) gauge returns Q_prev itself: the fixed point is the dominant
    invariant subspace of M, the same one the EVD projector keeps.  Without S
    the gauge alternates on negative eigenvalues and the iteration settles on
    a different subspace;
  * initial environment: C_0 = I_chi, T_0[a, u, b] = delta_ab t_u with
    t_u = sum_{v, w} a[u, (v v), (w w)] (both other legs closed by vec(I_D));
  * C and T are normalised to unit Frobenius norm after every step;
  * convergence: delta = || s_t - s_{t-1} ||_2 of the unit-norm, descending
    singular values of C.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ctm_oracle.c")
_LIB = os.path.join(_HERE, "libctm_oracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile ctm_oracle.c into a shared library next to it (plain gcc, -O2, OpenMP
    where the compiler has it; the results do not depend on the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            sig = {
                "orc_set_threads": (I, [I]),
                "orc_c3v_project": (None, [I, I, P, P]),
                "orc_frobenius": (ctypes.c_double, [ctypes.c_long, P]),
                "orc_double_layer": (None, [I, I, P, P, P]),
                "orc_matmul": (None, [I, I, I, P, P, P]),
                "orc_matmul_tn": (None, [I, I, I, P, P, P]),
                "orc_enlarged_corner": (None, [I, I, P, P, P, P, P]),
                "orc_householder_qr": (None, [I, I, P, P, P]),
                "orc_corner_update": (ctypes.c_double, [I, I, P, P, P]),
                "orc_corner_from_r": (ctypes.c_double, [I, P, P, P]),
                "orc_edge_update": (ctypes.c_double, [I, I, P, P, P, P, P]),
                "orc_sym_eig": (I, [I, P, P, P]),
                "orc_corner_spectrum": (None, [I, P, P]),
                "orc_evd_projector": (None, [I, I, P, P]),
                "orc_rho": (None, [I, I, I, P, P, P, P, P]),
                "orc_transfer_apply": (None, [I, I, P, P, P, P, P]),
                "orc_transfer_matrix": (None, [I, I, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(x: np.ndarray):
    assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def set_threads(nthreads: int = 0) -> int:
    """Threads of the oracle's parallel loops (<= 0: all cores); returns the count in effect."""
    return int(_load().orc_set_threads(int(nthreads)))


# --- single steps (each mirrors one row of the hot path) -------------------

def c3v_project(A: np.ndarray) -> np.ndarray:
    """a0 (Appendix A): average over the six permutations of the virtual legs."""
    A = _c(A)
    d, D = A.shape[0], A.shape[1]
    out = np.empty_like(A)
    _load().orc_c3v_project(d, D, _p(A), _p(out))
    return out


def prepare_site(A: np.ndarray, symmetrize: bool = True) -> np.ndarray:
    """a0: C3v projection followed by unit Frobenius norm (or A unchanged)."""
    A = _c(A)
    if not symmetrize:
        return A.copy()
    As = c3v_project(A)
    return As / _load().orc_frobenius(As.size, _p(As))


def double_layer(A: np.ndarray, B: np.ndarray | None = None) -> np.ndarray:
    """a1 (Fig. 1b): a[(ii'),(jj'),(kk')] = sum_s A[s,i,j,k] B[s,i',j',k']."""
    A = _c(A)
    B = A if B is None else _c(B)
    d, D = A.shape[0], A.shape[1]
    D2 = D * D
    a = np.empty((D2, D2, D2))
    _load().orc_double_layer(d, D, _p(A), _p(B), _p(a))
    return a


def enlarged_corner(C, T, aB, aA) -> np.ndarray:
    """a2 (Fig. 3c): M[(a,y),(b,x)] = sum T[a,u,g] C[g,h] T[b,l,h] aB[u,l,z] aA[z,x,y]."""
    C, T, aB, aA = _c(C), _c(T), _c(aB), _c(aA)
    chi, D2 = T.shape[0], T.shape[1]
    M = np.empty((chi * D2, chi * D2))
    _load().orc_enlarged_corner(chi, D2, _p(C), _p(T), _p(aB), _p(aA), _p(M))
    return M


def matmul(A, B) -> np.ndarray:
    A, B = _c(A), _c(B)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = np.empty((m, n))
    _load().orc_matmul(m, k, n, _p(A), _p(B), _p(C))
    return C


def householder_qr(Y):
    """a4 (Fig. 3d): thin Householder QR with diag(R) >= 0."""
    Y = _c(Y)
    n, k = Y.shape
    Q = np.empty((n, k))
    R = np.empty((k, k))
    _load().orc_householder_qr(n, k, _p(Y), _p(Q), _p(R))
    return Q, R


def corner_update(M, Q) -> np.ndarray:
    """a5 (Fig. 3a): C' = sym(Q^T M Q) / ||.||_F."""
    M, Q = _c(M), _c(Q)
    n, chi = Q.shape
    Cn = np.empty((chi, chi))
    _load().orc_corner_update(n, chi, _p(M), _p(Q), _p(Cn))
    return Cn


def corner_from_r(R, Cprev) -> np.ndarray:
    """Cheap variant of a5: C' = sym(R S) / ||.||_F, S = diag(sgn Cprev_jj), from the QR
    factor R of Y = M Q_prev S (R S = Q^T M Q_prev, equal to Q^T M Q at a fixed point)."""
    R, Cprev = _c(R), _c(Cprev)
    chi = R.shape[0]
    Cn = np.empty((chi, chi))
    _load().orc_corner_from_r(chi, _p(R), _p(Cprev), _p(Cn))
    return Cn


def edge_update(T, aB, aA, Q) -> np.ndarray:
    """a6 (Fig. 3b): T'[i,x,j] = sum Q[(a,y),i] T[a,u,g] aB[u,w,z] aA[z,x,y] Q[(g,w),j], normalised."""
    T, aB, aA, Q = _c(T), _c(aB), _c(aA), _c(Q)
    chi, D2 = T.shape[0], T.shape[1]
    Tn = np.empty_like(T)
    _load().orc_edge_update(chi, D2, _p(T), _p(aB), _p(aA), _p(Q), _p(Tn))
    return Tn


def sym_eig(S):
    """Cyclic Jacobi eigen-decomposition of a symmetric matrix (unsorted)."""
    S = _c(S)
    n = S.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    _load().orc_sym_eig(n, _p(S), _p(w), _p(V))
    return w, V


def corner_spectrum(C) -> np.ndarray:
    """a7: singular values of the symmetric corner, descending, unit 2-norm."""
    C = _c(C)
    s = np.empty(C.shape[0])
    _load().orc_corner_spectrum(C.shape[0], _p(C), _p(s))
    return s


def evd_projector(M, chi) -> np.ndarray:
    """Conventional EVD projector (Fig. 3c): top-|eigenvalue| eigenvectors of M."""
    M = _c(M)
    n = M.shape[0]
    P = np.empty((n, chi))
    _load().orc_evd_projector(n, chi, _p(M), _p(P))
    return P


def rho_bond(A, C, T, Q) -> np.ndarray:
    """a8 (Eq. 1, Fig. 5b): two-site reduced density matrix of the apex radial bond."""
    A, C, T, Q = _c(A), _c(C), _c(T), _c(Q)
    d, D = A.shape[0], A.shape[1]
    chi = C.shape[0]
    rho = np.empty((d * d, d * d))
    _load().orc_rho(d, D, chi, _p(A), _p(C), _p(T), _p(Q), _p(rho))
    return rho


def transfer_apply(T, aB, aA, v) -> np.ndarray:
    """f2 (Sec. II.C, Fig. 4a): TM v for the transfer matrix
    TM[(a,y,b),(g,w,h)] = sum T[a,u,g] aB[u,w,z] aA[z,x,y] T[b,x,h] (one Bravais step)."""
    T, aB, aA, v = _c(T), _c(aB), _c(aA), _c(v)
    chi, D2 = T.shape[0], T.shape[1]
    out = np.empty(chi * D2 * chi)
    _load().orc_transfer_apply(chi, D2, _p(T), _p(aB), _p(aA), _p(v.reshape(-1)), _p(out))
    return out


def transfer_matrix(T, aB, aA) -> np.ndarray:
    """The dense transfer matrix (chi D2 chi square; small cases)."""
    T, aB, aA = _c(T), _c(aB), _c(aA)
    chi, D2 = T.shape[0], T.shape[1]
    N = chi * D2 * chi
    TM = np.empty((N, N))
    _load().orc_transfer_matrix(chi, D2, _p(T), _p(aB), _p(aA), _p(TM))
    return TM


def transfer_spectrum(T, aB, aA, nev: int = 3, dense_max: int = 4096):
    """Magnitudes of the nev largest-magnitude eigenvalues of the transfer matrix,
    normalised by the largest (lambda_i = |lambda_i'| / |lambda_0'|, Sec. II.C), the
    correlation length xi = -1 / ln lambda_1 in Bravais steps and the gap
    ln(lambda_1 / lambda_2) of the FCLS extrapolation (Eq. 3).  LAPACK's general
    eigenvalues on the dense matrix when it is small, else ARPACK on transfer_apply."""
    chi, D2 = T.shape[0], T.shape[1]
    N = chi * D2 * chi
    if N <= dense_max:
        w = np.linalg.eigvals(transfer_matrix(T, aB, aA))
    else:
        import scipy.sparse.linalg as sla
        op = sla.LinearOperator((N, N), matvec=lambda v: transfer_apply(T, aB, aA, v), dtype=np.float64)
        w = sla.eigs(op, k=max(nev, 3) + 2, which="LM", tol=1e-13, return_eigenvectors=False)
    lam = np.sort(np.abs(w))[::-1][:nev]
    lam = lam / lam[0]
    xi = -1.0 / np.log(lam[1]) if lam[1] > 0.0 else 0.0
    gap = np.log(lam[1] / lam[2]) if nev >= 3 and lam[2] > 0.0 else float("inf")
    return lam, xi, gap


def bond_energies(rho, h):
    """e_a = tr(rho h_a) for a = x, y, z; E_site = (1/2) sum_a e_a (3 bonds per site, 2 sites per bond)."""
    h = np.asarray(h, dtype=np.float64)
    e = np.array([float(np.sum(rho * h[a].T)) for a in range(3)])
    return e, 0.5 * float(np.sum(e))


# --- the iteration ----------------------------------------------------------

class OracleCTM:
    """QR-based (or, for cross-checks, EVD-based) C3v CTMRG on one site tensor."""

    def __init__(self, A, chi: int, symmetrize: bool = True, projector: str = "qr", corner: str = "qmq"):
        self.corner = corner          # "qmq": C' = sym(Q^T M Q); "r": the cheap variant sym(R S)
        self.A = prepare_site(A, symmetrize)
        self.d, self.D = self.A.shape[0], self.A.shape[1]
        self.D2 = self.D * self.D
        self.chi = int(chi)
        self.n = self.chi * self.D2
        self.projector = projector
        self.a = double_layer(self.A)
        D, D2, chi = self.D, self.D2, self.chi
        diag = np.array([v * D + v for v in range(D)])
        t = self.a[:, diag][:, :, diag].sum(axis=(1, 2))
        self.C = np.eye(chi)
        self.T = np.zeros((chi, D2, chi))
        for al in range(chi):
            self.T[al, :, al] = t
        self.Q = np.zeros((self.n, chi))
        self.Q[np.arange(chi), np.arange(chi)] = 1.0
        self.s = corner_spectrum(self.C)
        self.last = {}
        self.steps = 0

    def set_env(self, C, T, Q):
        self.C, self.T, self.Q = _c(C).copy(), _c(T).copy(), _c(Q).copy()
        self.s = corner_spectrum(self.C)

    def warm_start(self) -> np.ndarray:
        """Q_prev S, S = diag(sgn C_ii) with sgn(0) = +1."""
        S = np.where(np.diag(self.C) < 0.0, -1.0, 1.0)
        return self.Q * S[None, :]

    def step(self) -> float:
        M = enlarged_corner(self.C, self.T, self.a, self.a)
        if self.projector == "qr":
            Y = matmul(M, self.warm_start())
            Q, R = householder_qr(Y)
        else:
            Y, R = None, None
            Q = evd_projector(M, self.chi)
        if self.corner == "r" and self.projector == "qr":
            Cn = corner_from_r(R, self.C)
        else:
            Cn = corner_update(M, Q)
        Tn = edge_update(self.T, self.a, self.a, Q)
        s = corner_spectrum(Cn)
        delta = float(np.sqrt(np.sum((s - self.s) ** 2)))
        self.last = {"M": M, "Y": Y, "Q": Q, "R": R, "C": Cn, "T": Tn}
        self.C, self.T, self.Q, self.s = Cn, Tn, Q, s
        self.steps += 1
        return delta

    def converge(self, max_steps: int, tol: float):
        delta = float("inf")
        for k in range(max_steps):
            delta = self.step()
            if delta < tol:
                return k + 1, delta
        return max_steps, delta

    def projector_for_energy(self):
        """The projector a further step would use: QR of M Q_prev (or the EVD projector)."""
        M = enlarged_corner(self.C, self.T, self.a, self.a)
        if self.projector == "qr":
            return householder_qr(matmul(M, self.warm_start()))[0]
        return evd_projector(M, self.chi)

    def rho(self):
        return rho_bond(self.A, self.C, self.T, self.projector_for_energy())

    def energy(self, h):
        return bond_energies(self.rho(), h)

    def transfer_spectrum(self, nev: int = 3):
        """f2: leading transfer-matrix eigenvalues of the current environment, xi, gap."""
        return transfer_spectrum(self.T, self.a, self.a, nev)
