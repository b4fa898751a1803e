"""Error bounds of the split-BF16 step, derived from the engine's per-contraction
truncation bound (test infrastructure; no expected values are computed here).

One split contraction C = A B with n_split = T slices per operand differs from the
exact product by at most  beta K max_k|A_mk| max_k|B_kn|,  beta = (T + 1) 2^(-8T)
(the dropped slice pairs; the engine's own tests check this bound).  An error
already carried by an operand adds |A| e_B + e_A |B| (first order).  The chains
below follow the step's contractions in the engine's order with the magnitudes of
the oracle's own operands.

The projector comes from the FP64 Householder QR of Y; for Y + dY = (Q + dQ)(R + dR)
the first-order perturbation of the thin QR gives
    ||dQ||_F <= sqrt(2) ||R^-1||_2 ||dY||_F,   ||dR||_F <= sqrt(2) kappa_2(R) ||dY||_F
(from Q^T dY R^-1 = Q^T dQ + dR R^-1 with Q^T dQ skew on the leading block and
dR R^-1 upper triangular).  The first `lead` columns of Q and rows of R depend only
on the first `lead` columns of Y, so R is restricted to that block.  A normalised
X / ||X||_F moves by at most 2 ||dX||_F / ||X||_F.
"""
import numpy as np


def beta(T):
    return (T + 1) * 2.0 ** (-8 * T)


def gemm_err(A, B, T, eA=None, eB=None):
    """Elementwise bound of the split product A B (2-D operands)."""
    K = A.shape[1]
    e = beta(T) * K * np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(B), axis=0)[None, :]
    if eA is not None:
        e = e + eA @ np.abs(B)
    if eB is not None:
        e = e + np.abs(A) @ eB
    return e


def enlarged_corner_err(C, T, a, Tn):
    """Bound on |M_split - M| for the chain W = T C, X' = W T^T, Y1 = X' a, M = Y1 a."""
    chi, D2 = T.shape[0], T.shape[1]
    n = chi * D2
    Tm = T.reshape(n, chi)                        # rows (a, u), K = g
    W = Tm @ C
    eW = gemm_err(Tm, C, Tn)
    X = W @ Tm.T                                  # rows (a, u), cols (b, l)
    eX = gemm_err(W, Tm.T, Tn, eA=eW)
    # Y1[(a,b)][z] = sum_{(u,l)} X'[(a,b),(u,l)] a[(u,l), z]
    Xr = X.reshape(chi, D2, chi, D2).transpose(0, 2, 1, 3).reshape(chi * chi, D2 * D2)
    eXr = eX.reshape(chi, D2, chi, D2).transpose(0, 2, 1, 3).reshape(chi * chi, D2 * D2)
    aB = a.reshape(D2 * D2, D2)
    Y1 = Xr @ aB
    eY1 = gemm_err(Xr, aB, Tn, eA=eXr)
    # M[(a,y)][(b,x)] = sum_z Y1[(a,b), z] a[z, x, y]
    aA = a.reshape(D2, D2 * D2)
    eMr = gemm_err(Y1, aA, Tn, eA=eY1)            # rows (a, b), cols (x, y)
    return eMr.reshape(chi, chi, D2, D2).transpose(0, 3, 1, 2).reshape(n, n)


def edge_chain_err(T, a, Q, Tn):
    """Bound on |T'_raw split - T'_raw| from the edge chain's own truncations (Q exact)."""
    chi, D2 = T.shape[0], T.shape[1]
    n = chi * D2
    Tm = T.reshape(n, chi)
    Bq = Q.reshape(chi, D2, chi).transpose(0, 2, 1).reshape(chi, chi * D2)   # [g][(j, w)]
    H1 = Tm @ Bq                                   # rows (a, u), cols (j, w)
    eH1 = gemm_err(Tm, Bq, Tn)
    H1r = H1.reshape(chi, D2, chi, D2).transpose(0, 2, 1, 3).reshape(chi * chi, D2 * D2)
    eH1r = eH1.reshape(chi, D2, chi, D2).transpose(0, 2, 1, 3).reshape(chi * chi, D2 * D2)
    aB = a.reshape(D2 * D2, D2)
    H2 = H1r @ aB                                  # rows (a, j), K (u, w)
    eH2 = gemm_err(H1r, aB, Tn, eA=eH1r)
    aA = a.reshape(D2, D2 * D2)
    H3 = H2 @ aA                                   # rows (a, j), cols (x, y)
    eH3 = gemm_err(H2, aA, Tn, eA=eH2)
    # T'[i][(x, j)] = sum_{(a, y)} Q[(a,y), i] H3'[(a,y),(x,j)]
    H3r = H3.reshape(chi, chi, D2, D2).transpose(0, 3, 2, 1).reshape(n, D2 * chi)
    eH3r = eH3.reshape(chi, chi, D2, D2).transpose(0, 3, 2, 1).reshape(n, D2 * chi)
    return gemm_err(Q.T, H3r, Tn, eB=eH3r)


def edge_operator_fro(T, a):
    """||K||_F of T'_raw[i,x,j] = sum Q[(a,y),i] K[(a,y), x, (g,w)] Q[(g,w),j],
    K = T a a, from P[u][(w,x,y)] = sum_z a[u,w,z] a[z,x,y]: ||K||_F^2 = tr(Tm (P P^T) Tm^T)
    with Tm[(a,g)][u] = T[a,u,g]."""
    chi, D2 = T.shape[0], T.shape[1]
    P = np.einsum("uwz,zxy->uwxy", a, a).reshape(D2, -1)
    G = P @ P.T
    Tm = T.transpose(0, 2, 1).reshape(chi * chi, D2)
    return float(np.sqrt(max(np.einsum("iu,uv,iv->", Tm, G, Tm), 0.0)))


def qr_bounds(dY_fro, Y, R, lead):
    """First-order bounds on ||dQ[:, :lead]||_F and ||dR[:lead]||_F (so also on the
    largest entry of each) for a perturbation
    dY of the reduced corner, plus the backward error of the two FP64 Householder
    factorisations being compared (each ||dY_j|| <= gamma ||Y_j||, gamma = n chi u,
    u = 2^-53; Higham, Accuracy and Stability of Numerical Algorithms, Thm 19.4)."""
    n, chi = Y.shape
    gamma = n * chi * 2.0 ** -53
    dY = dY_fro + 2.0 * gamma * float(np.linalg.norm(Y[:, :lead]))
    sv = np.linalg.svd(R[:lead, :lead], compute_uv=False)
    dQ = np.sqrt(2.0) * dY / sv[-1]
    dR = np.sqrt(2.0) * (sv[0] / sv[-1]) * dY
    return dQ, dR


def qr_column_bounds(dY, Y, R, lead):
    """Per-column version of qr_bounds: column j of Q (and of R) depends only on the
    first j + 1 columns of Y, so its bound uses R[:j+1, :j+1] and dY[:, :j+1].
    Returns arrays bq[j] >= ||dQ[:, j]||_2 and br[j] >= ||dR[:j+1, j]||_2 for j < lead."""
    n, chi = Y.shape
    gamma = n * chi * 2.0 ** -53
    bq = np.empty(lead)
    br = np.empty(lead)
    for j in range(lead):
        dYj = float(np.linalg.norm(dY[:, :j + 1])) + 2.0 * gamma * float(np.linalg.norm(Y[:, :j + 1]))
        sv = np.linalg.svd(R[:j + 1, :j + 1], compute_uv=False)
        bq[j] = np.sqrt(2.0) * dYj / sv[-1]
        br[j] = np.sqrt(2.0) * (sv[0] / sv[-1]) * dYj
    return bq, br


def corner_bound(M, Q, dM_fro, dQ, Tn):
    """Bound on ||dC'||_F for C' = sym(Q^T M Q)/||.||_F: perturbations dM and dQ
    (Frobenius norms)
    (||Q^T dM Q||_F <= ||dM||_F, ||dQ^T M Q||_F <= ||M||_F ||dQ||_F) plus the
    truncation of the split contractions M Q and Q^T (M Q)."""
    MQ = M @ Q
    eMQ = gemm_err(M, Q, Tn)
    eCr = gemm_err(Q.T, MQ, Tn, eB=eMQ)
    Cr = Q.T @ MQ
    Csym = 0.5 * (Cr + Cr.T)
    dCr = float(np.linalg.norm(eCr)) + dM_fro + 2.0 * float(np.linalg.norm(M)) * dQ
    return 2.0 * dCr / float(np.linalg.norm(Csym))


def edge_bound(T, a, Q, dQ, Tn):
    """Bound on ||dT'||_F for T' = Q^T (T a a) Q / ||.||_F: the perturbation dQ (Frobenius) on both
    sides (2 ||K||_F ||dQ||_F) plus the edge chain's own truncations."""
    chi, D2 = T.shape[0], T.shape[1]
    eT = edge_chain_err(T, a, Q, Tn)
    Traw = np.einsum("ayi,ayxj->ixj", Q.reshape(chi, D2, chi),
                     np.einsum("aug,uwz,zxy,gwj->ayxj", T, a, a, Q.reshape(chi, D2, chi), optimize=True),
                     optimize=True)
    dTraw = float(np.linalg.norm(eT)) + 2.0 * edge_operator_fro(T, a) * dQ
    return 2.0 * dTraw / float(np.linalg.norm(Traw))
