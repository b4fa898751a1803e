"""CPU reference gradient: PyTorch float64 autograd of an einsum restatement of the
QR-CTMRG forward (test infrastructure, written independently of the CUDA adjoint).

Follows the same readings as the oracle: C3v projection + unit norm, double
layer, enlarged corner of the radial-dimer sector, reduced corner
Y = M Q_prev diag(sgn C_ii), thin QR with diag(R) >= 0, C' = sym(Q^T M Q)/|.|,
T' = Q^T (T a a) Q/|.|, and the bond energy rho = tr(Ch^5 Q^T M_oo Q)/tr(Ch^6).
The environment entering the tracked steps is a constant (no gradient).
"""
import torch


def project(Araw):
    P = (Araw + Araw.permute(0, 1, 3, 2) + Araw.permute(0, 2, 1, 3) + Araw.permute(0, 2, 3, 1) +
         Araw.permute(0, 3, 1, 2) + Araw.permute(0, 3, 2, 1)) / 6.0
    return P / torch.linalg.norm(P)


def layer(K, B):
    D = K.shape[1]
    return torch.einsum("sijk,slmn->iljmkn", K, B).reshape(D * D, D * D, D * D)


def enlarged_corner(C, T, aB, aA):
    chi, D2 = T.shape[0], T.shape[1]
    X = torch.einsum("aug,gh,blh->aulb", T, C, T)
    return torch.einsum("aulb,ulz,zxy->aybx", X, aB, aA).reshape(chi * D2, chi * D2)


def qr_gauge(Y):
    Q, R = torch.linalg.qr(Y, mode="reduced")
    s = torch.where(torch.diagonal(R) < 0, -1.0, 1.0).to(Y.dtype)
    return Q * s[None, :], R * s[:, None]


def projector(C, T, Qp, a):
    M = enlarged_corner(C, T, a, a)
    S = torch.where(torch.diagonal(C) < 0, -1.0, 1.0).to(C.dtype)
    Q, R = qr_gauge(M @ (Qp * S[None, :]))
    return M, Q


def step(C, T, Qp, a):
    chi, D2 = T.shape[0], T.shape[1]
    M, Q = projector(C, T, Qp, a)
    Cr = Q.T @ M @ Q
    Cs = 0.5 * (Cr + Cr.T)
    Cn = Cs / torch.linalg.norm(Cs)
    Q4 = Q.reshape(chi, D2, chi)
    Tn = torch.einsum("ayi,aug,uwz,zxy,gwj->ixj", Q4, T, a, a, Q4)
    return Cn, Tn / torch.linalg.norm(Tn), Q


def energy(C, T, Qp, A, h):
    d = A.shape[0]
    a = layer(A, A)
    M, Q = projector(C, T, Qp, a)
    Cr = Q.T @ M @ Q
    Ch = 0.5 * (Cr + Cr.T)
    Ch = Ch / torch.linalg.norm(Ch)
    P5 = torch.linalg.matrix_power(Ch, 5)
    raw = torch.zeros((d * d, d * d), dtype=A.dtype)
    rows = []
    for sA in range(d):
        for sB in range(d):
            row = []
            for tA in range(d):
                for tB in range(d):
                    bA = layer(A[sA:sA + 1], A[tA:tA + 1])
                    bB = layer(A[sB:sB + 1], A[tB:tB + 1])
                    Moo = enlarged_corner(C, T, bB, bA)
                    row.append(torch.trace(P5 @ (Q.T @ Moo @ Q)))
            rows.append(torch.stack(row))
    raw = torch.stack(rows)
    rho = raw / torch.trace(raw)
    e = torch.stack([torch.sum(rho * h[k].T) for k in range(3)])
    return 0.5 * e.sum()


def energy_and_grad(Araw, env, h, k_tracked):
    """E and dE/dAraw through k_tracked steps from the constant environment env = (C, T, Q)."""
    Araw = torch.as_tensor(Araw, dtype=torch.float64).clone().requires_grad_(True)
    C, T, Q = (torch.as_tensor(x, dtype=torch.float64) for x in env)
    h = torch.as_tensor(h, dtype=torch.float64)
    A = project(Araw)
    a = layer(A, A)
    for _ in range(k_tracked):
        C, T, Q = step(C, T, Q, a)
    E = energy(C, T, Q, A, h)
    (g,) = torch.autograd.grad(E, Araw)
    return float(E.detach()), g.numpy()
