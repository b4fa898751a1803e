"""Seeded synthetic inputs for the honeycomb QR-CTMRG hot path.

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It holds input generation only -- random site tensors, bond
Hamiltonians, a classical-Ising site tensor and the workload table -- and none
of the CTMRG arithmetic (no symmetrisation, no double layer, no contraction).

The paper's workloads are optimised Heisenberg / Kitaev iPEPS tensors (Sec. III)
which are not available; seeded uniform[-1, 1] tensors of the same shapes stand
in for them.  The Hamiltonian is the Kitaev-Heisenberg model of Eq. (4),
H = sum_<ij>_a K S^a_i S^a_j + J sum_<ij> S_i . S_j, with S = sigma / 2 for
spin-1/2 (Sec. III.A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "random_site_tensor",
    "product_site_tensor",
    "perturbed_product_site_tensor",
    "ising_site_tensor",
    "spin_matrices",
    "bond_hamiltonians",
    "Workload",
    "WORKLOADS",
    "batch_workload",
]


def random_site_tensor(d: int, D: int, seed: int) -> np.ndarray:
    """Raw site tensor A[s, i, j, k] with entries uniform in [-1, 1].

    Layout: float64, shape (d, D, D, D), row-major (s slowest).  The
    C3v (A1) projection and the Frobenius normalisation are part of the method
    and are *not* applied here.
    """
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(d, D, D, D)).astype(np.float64)


def product_site_tensor(v) -> np.ndarray:
    """D = 1 site tensor A[s, 0, 0, 0] = v[s] (a product state |v> on every site)."""
    v = np.asarray(v, dtype=np.float64)
    return v.reshape(-1, 1, 1, 1).copy()


def perturbed_product_site_tensor(v, D: int, eps: float, seed: int) -> np.ndarray:
    """Product state |v> on every site plus a small seeded perturbation.

    A[s, i, j, k] = v[s] delta_{i0} delta_{j0} delta_{k0} + eps * U[s, i, j, k] with U
    uniform in [-1, 1] from ``default_rng(seed)``.  Its correlations are short, so
    the corner spectrum falls off fast: at D = 6 the 72nd unit-norm
    corner singular value is ~1e-12 at eps = 0.002, and a chi = 72 environment
    converges to delta < 1e-10 in a few steps (a random tensor at D = 6 has no spectral gap at
    chi = 72 and does not converge).  Not projected or normalised here.
    """
    v = np.asarray(v, dtype=np.float64)
    rng = np.random.default_rng(seed)
    A = eps * rng.uniform(-1.0, 1.0, size=(v.size, D, D, D))
    A[:, 0, 0, 0] += v
    return A


def coherent_state(d: int, direction) -> np.ndarray:
    """Spin-S coherent state |S, m = S> along a unit vector (theta, phi), in the S^z basis
    m = S, S-1, ..., -S: c_m = sqrt(binom(2S, S-m)) cos(theta/2)^(S+m) sin(theta/2)^(S-m)
    e^{i (S-m) phi}.  The spin-1/2 state along (1,1,1)/sqrt 3 is the one the three-fold
    spin rotation about that axis leaves unchanged (the seed of the complex workloads)."""
    x, y, z = (float(c) for c in direction)
    r = math.sqrt(x * x + y * y + z * z)
    theta, phi = math.acos(z / r), math.atan2(y, x)
    twoS = d - 1
    c = np.zeros(d, dtype=np.complex128)
    for k in range(d):                     # k = S - m
        c[k] = (math.sqrt(math.comb(twoS, k)) * math.cos(theta / 2) ** (twoS - k) * math.sin(theta / 2) ** k
                * np.exp(1j * k * phi))
    return c


def complex_perturbed_product_site_tensor(v, D: int, eps: float, seed: int) -> np.ndarray:
    """Complex counterpart of perturbed_product_site_tensor: A = v (x) e_000 + eps (U + i V),
    U and V uniform in [-1, 1] from ``default_rng(seed)``.  Not projected or normalised."""
    v = np.asarray(v, dtype=np.complex128)
    rng = np.random.default_rng(seed)
    A = eps * (rng.uniform(-1.0, 1.0, size=(v.size, D, D, D)) + 1j * rng.uniform(-1.0, 1.0, size=(v.size, D, D, D)))
    A[:, 0, 0, 0] += v
    return A


def random_complex_site_tensor(d: int, D: int, seed: int) -> np.ndarray:
    """A[s, i, j, k] = U + i V, U and V uniform in [-1, 1] from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(d, D, D, D)) + 1j * rng.uniform(-1.0, 1.0, size=(d, D, D, D))


def ising_site_tensor(beta: float) -> np.ndarray:
    """Site tensor whose norm network is the classical Ising model on the honeycomb lattice.

    A[s; i, j, k] = W[s, i] W[s, j] W[s, k] with (W W^T)[s, t] = exp((beta/2) sigma_s sigma_t),
    sigma = (+1, -1).  Contracting two double-layer tensors over a bond gives
    (W W^T)[s, t]^2 = exp(beta sigma_s sigma_t), so <Psi|Psi> is the honeycomb
    Ising partition function and 4 <S^z S^z> on a bond is the nearest-neighbour
    spin correlation.  d = D = 2, real, symmetric in its three virtual legs.
    """
    # (W W^T) = [[e^{b/2}, e^{-b/2}], [e^{-b/2}, e^{b/2}]] has eigenvalues
    # 2 cosh(b/2) (vector (1,1)/sqrt2) and 2 sinh(b/2) (vector (1,-1)/sqrt2).
    l0 = 2.0 * math.cosh(beta / 2.0)
    l1 = 2.0 * math.sinh(beta / 2.0)
    if l1 <= 0.0:
        raise ValueError("beta must be positive")
    r = 1.0 / math.sqrt(2.0)
    W = np.array([[r * math.sqrt(l0), r * math.sqrt(l1)],
                  [r * math.sqrt(l0), -r * math.sqrt(l1)]])
    return np.einsum("si,sj,sk->sijk", W, W, W)


def spin_matrices(d: int = 2):
    """Spin-S operators (S^x, S^y, S^z) for d = 2S + 1 in the S^z basis (m = S, S-1, ...)."""
    S = (d - 1) / 2.0
    m = S - np.arange(d)
    Sz = np.diag(m).astype(np.complex128)
    Sp = np.zeros((d, d), dtype=np.complex128)
    for k in range(1, d):
        # <m+1| S^+ |m> = sqrt(S(S+1) - m(m+1)), with row k-1 holding m+1
        mm = m[k]
        Sp[k - 1, k] = math.sqrt(S * (S + 1) - mm * (mm + 1))
    Sx = (Sp + Sp.conj().T) / 2.0
    Sy = (Sp - Sp.conj().T) / 2.0j
    return Sx, Sy, Sz


def bond_hamiltonians(K: float, J: float, d: int = 2, rotate_b: bool = False) -> np.ndarray:
    """Bond operators h_a = K S^a S^a + J S.S for a = x, y, z (Eq. 4), as real d^2 x d^2 matrices.

    Row index (s_A, s_B) = s_A * d + s_B, column index likewise: h[(s t), (s' t')] =
    <s t| h |s' t'>.  ``rotate_b`` applies the pi-rotation about y on the B site
    used for the uniform Heisenberg ansatz (Sec. III.B): S^x_B -> -S^x_B,
    S^z_B -> -S^z_B.
    """
    Sx, Sy, Sz = spin_matrices(d)
    sgn = (-1.0, 1.0, -1.0) if rotate_b else (1.0, 1.0, 1.0)
    ops = (Sx, Sy, Sz)
    pair = [sgn[a] * np.kron(ops[a], ops[a]) for a in range(3)]
    heis = pair[0] + pair[1] + pair[2]
    hs = []
    for a in range(3):
        h = K * pair[a] + J * heis
        if np.max(np.abs(h.imag)) > 1e-14:
            raise ValueError("bond operator is not real")
        hs.append(h.real)
    return np.ascontiguousarray(np.stack(hs), dtype=np.float64)


@dataclass
class Workload:
    """One single-instance CTMRG workload (d, D, chi, Hamiltonian, seed)."""
    name: str
    d: int
    D: int
    chi: int
    K: float
    J: float
    seed: int
    steps: int
    tol: float = 1e-10
    precision: str = "fp64"
    note: str = ""
    eps: float = 0.0          # > 0: perturbed product state (perturbed_product_site_tensor)
    irrep: str = "A1"         # "E": complex tensor for the complex representation of C3v

    @property
    def D2(self) -> int:
        return self.D * self.D

    @property
    def n(self) -> int:
        return self.chi * self.D * self.D

    def site_tensor(self) -> np.ndarray:
        if self.irrep == "E":
            if self.eps > 0.0:
                return complex_perturbed_product_site_tensor(coherent_state(self.d, (1.0, 1.0, 1.0)), self.D,
                                                             self.eps, self.seed)
            return random_complex_site_tensor(self.d, self.D, self.seed)
        if self.eps > 0.0:
            return perturbed_product_site_tensor(_PRODUCT_V[:self.d] / np.linalg.norm(_PRODUCT_V[:self.d]),
                                                 self.D, self.eps, self.seed)
        return random_site_tensor(self.d, self.D, self.seed)

    def hamiltonians(self) -> np.ndarray:
        return bond_hamiltonians(self.K, self.J, self.d)


_PHI = 0.3 * math.pi
_PRODUCT_V = np.array([0.8, 0.6, 0.0])

# The workloads: Heisenberg D=2/chi=8 (oracle-sized), Kitaev D=4/chi=32,
# Kitaev-Heisenberg D=6/chi=72 and D=8/chi=128 (phi = 0.3 pi), their converging
# near-product counterparts, and a 96-instance ragged batch.  Seeds are
# 1000 + index (5000 + i for the batch instances).
WORKLOADS = {
    "heis_D2_chi8": Workload("heis_D2_chi8", 2, 2, 8, 0.0, 1.0, 1000, 50,
                             note="Heisenberg J=1, 50 steps or delta<1e-10"),
    "kitaev_D4_chi32": Workload("kitaev_D4_chi32", 2, 4, 32, 1.0, 0.0, 1001, 200,
                                note="isotropic Kitaev K=1, 200 steps"),
    "kh_D6_chi72": Workload("kh_D6_chi72", 2, 6, 72, math.cos(_PHI), math.sin(_PHI), 1002, 200,
                            note="Kitaev-Heisenberg phi=0.3pi, enlarged corner 2592x2592"),
    "kh_D8_chi128": Workload("kh_D8_chi128", 2, 8, 128, math.cos(_PHI), math.sin(_PHI), 1003, 30,
                             note="Kitaev-Heisenberg phi=0.3pi, enlarged corner 8192x8192"),
    # converging stand-ins at the same sizes: product state (0.8, 0.6) plus a small
    # seeded perturbation (short correlations, fast-falling corner spectrum)
    "kitaev_D4_chi32_conv": Workload("kitaev_D4_chi32_conv", 2, 4, 32, 1.0, 0.0, 1004, 200, eps=0.005,
                                     note="isotropic Kitaev K=1, near-product state, converges to 1e-10"),
    "kh_D6_chi72_conv": Workload("kh_D6_chi72_conv", 2, 6, 72, math.cos(_PHI), math.sin(_PHI), 1005, 200,
                                 eps=0.002,
                                 note="Kitaev-Heisenberg phi=0.3pi, near-product state, converges to 1e-10"),
    "kh_D8_chi128_conv": Workload("kh_D8_chi128_conv", 2, 8, 128, math.cos(_PHI), math.sin(_PHI), 1006, 200,
                                  eps=0.002,
                                  note="Kitaev-Heisenberg phi=0.3pi, near-product state, D=8, chi=128"),
    # complex tensors for the E irrep of C3v (the Kitaev model's representation, ferromagnetic
    # K = -1 as in Sec. III.C): the spin-1/2 state along (1,1,1) plus a small complex
    # perturbation (converging), and random complex tensors (step parity)
    "kitaev_E_D4_chi32_conv": Workload("kitaev_E_D4_chi32_conv", 2, 4, 32, -1.0, 0.0, 1007, 200, eps=0.005,
                                       irrep="E", note="Kitaev K=-1, complex E-irrep tensor, near-product"),
    "kitaev_E_D6_chi64_conv": Workload("kitaev_E_D6_chi64_conv", 2, 6, 64, -1.0, 0.0, 1008, 200, eps=0.002,
                                       irrep="E", note="Kitaev K=-1, complex E-irrep tensor, near-product, "
                                                       "enlarged corner 2304x2304 complex"),
    "kitaev_E_D6_chi64": Workload("kitaev_E_D6_chi64", 2, 6, 64, -1.0, 0.0, 1009, 30, irrep="E",
                                  note="Kitaev K=-1, random complex E-irrep tensor"),
    "kitaev_E_D6_chi72_conv": Workload("kitaev_E_D6_chi72_conv", 2, 6, 72, -1.0, 0.0, 1010, 200, eps=0.002,
                                       irrep="E", note="Kitaev K=-1, complex E-irrep tensor, near-product, "
                                                       "enlarged corner 2592x2592 complex"),
    "kitaev_E_D6_chi72": Workload("kitaev_E_D6_chi72", 2, 6, 72, -1.0, 0.0, 1011, 30, irrep="E",
                                  note="Kitaev K=-1, random complex E-irrep tensor, the size of kh_D6_chi72"),
}
# Heisenberg D = 5 at growing chi, the sweep of the paper's per-iteration runtime figure
# (Sec. III.B, Fig. 4c: D = 5, chi from 120 up): seeds 1012 + index
for _i, _chi in enumerate((120, 240, 360, 480)):
    WORKLOADS[f"heis_D5_chi{_chi}"] = Workload(f"heis_D5_chi{_chi}", 2, 5, _chi, 0.0, 1.0, 1012 + _i, 3,
                                               note=f"Heisenberg J=1, D=5, chi={_chi}, n={25 * _chi}")


def batch_workload(n_inst: int = 96, seed0: int = 5000):
    """Ragged batch: D uniform in {3,4,5,6}, chi uniform in {24,32,...,72}, phi_i = 2 pi i / n."""
    rng = np.random.default_rng(seed0)
    Ds = rng.integers(3, 7, size=n_inst)
    chis = 24 + 8 * rng.integers(0, 7, size=n_inst)
    out = []
    for i in range(n_inst):
        phi = 2.0 * math.pi * i / n_inst
        out.append(Workload(f"batch_{i}", 2, int(Ds[i]), int(chis[i]), math.cos(phi), math.sin(phi),
                            seed0 + i, 30, precision="split"))
    return out
