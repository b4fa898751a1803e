"""Hand-written adjoint (ctm_grad) against an independent CPU reference gradient
(PyTorch float64 autograd of an einsum restatement, tests/torch_reference.py) and
against central finite differences of the FP64 oracle.

The environment entering the tracked steps is held fixed on every side: the
reference and the finite differences start the tracked steps from the oracle's
environment after the warm-up steps.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _gpu_grad(A, chi, h, warmup, k, precision="fp64"):
    from paper_2509_05090_gb300 import binding
    g = binding.CTM(A, chi, precision=precision, n_split=5)
    E, dA = g.ctm_grad(h, warmup=warmup, k_tracked=k)
    out = dA.cpu().numpy()
    g.close()
    return E, out


def _oracle_env_after(A, chi, warmup):
    ref = O.OracleCTM(A, chi)
    for _ in range(warmup):
        ref.step()
    return ref.C.copy(), ref.T.copy(), ref.Q.copy()


def _oracle_energy(A, chi, env, h, k):
    ref = O.OracleCTM(A, chi)
    ref.set_env(*env)
    for _ in range(k):
        ref.step()
    return ref.energy(h)[1]


@pytest.mark.parametrize("wl,warmup,k", [("heis_D2_chi8", 5, 3), ("kitaev_D4_chi32", 3, 2)])
def test_adjoint_matches_cpu_reference_gradient(ctm_lib, wl, warmup, k):
    import torch_reference as TR
    w = I.WORKLOADS[wl]
    A, h = w.site_tensor(), w.hamiltonians()
    E_gpu, g_gpu = _gpu_grad(A, w.chi, h, warmup, k)
    env = _oracle_env_after(A, w.chi, warmup)
    E_ref, g_ref = TR.energy_and_grad(A, env, h, k)
    assert abs(E_gpu - E_ref) <= 1e-10
    assert np.max(np.abs(g_gpu - g_ref)) <= 1e-7 * np.max(np.abs(g_ref))


def test_adjoint_matches_finite_differences(ctm_lib):
    w = I.WORKLOADS["heis_D2_chi8"]
    A, h = w.site_tensor(), w.hamiltonians()
    warmup, k, step = 5, 3, 1e-6
    E, g = _gpu_grad(A, w.chi, h, warmup, k)
    env = _oracle_env_after(A, w.chi, warmup)
    rng = np.random.default_rng(3)
    for _ in range(3):
        V = rng.standard_normal(A.shape)
        fd = (_oracle_energy(A + step * V, w.chi, env, h, k) - _oracle_energy(A - step * V, w.chi, env, h, k)) / (2 * step)
        assert abs(fd - np.sum(g * V)) <= 1e-6 * max(1.0, abs(fd))


def test_autograd_function_backward(ctm_lib):
    import torch
    from paper_2509_05090_gb300.autograd import ctm_energy
    w = I.WORKLOADS["heis_D2_chi8"]
    A = torch.from_numpy(w.site_tensor()).cuda().requires_grad_(True)
    h = torch.from_numpy(w.hamiltonians()).cuda()
    E = ctm_energy(A, w.chi, h, warmup=5, k_tracked=3)
    (gA,) = torch.autograd.grad(2.0 * E, A)
    E2, g2 = _gpu_grad(w.site_tensor(), w.chi, w.hamiltonians(), 5, 3)
    assert abs(float(E.detach()) - E2) <= 1e-12
    assert np.max(np.abs(gA.cpu().numpy() - 2.0 * g2)) <= 1e-10 * np.max(np.abs(g2))


def test_adjoint_long_tracking_matches_cpu_reference(ctm_lib):
    """k = 12 tracked steps on the converging D = 2 workload."""
    import torch_reference as TR
    w = I.WORKLOADS["heis_D2_chi8"]
    A, h = w.site_tensor(), w.hamiltonians()
    E_gpu, g_gpu = _gpu_grad(A, w.chi, h, 10, 12)
    env = _oracle_env_after(A, w.chi, 10)
    E_ref, g_ref = TR.energy_and_grad(A, env, h, 12)
    assert abs(E_gpu - E_ref) <= 1e-10
    assert np.max(np.abs(g_gpu - g_ref)) <= 1e-7 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("k", [1, 2])
def test_adjoint_full_size_d8_chi128_directional(ctm_lib, k):
    """D = 8, chi = 128: consistent with a central difference of the GPU forward
    along one direction (a property at any size).  Short tracking: this random
    state does not converge, and through many unconverged steps the derivative
    is dominated by the growth of perturbations, not by the adjoint."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["kh_D8_chi128"]
    A, h = w.site_tensor(), w.hamiltonians()
    E, g = _gpu_grad(A, w.chi, h, 2, k)
    assert np.all(np.isfinite(g))
    rng = np.random.default_rng(8)
    V = rng.standard_normal(A.shape)
    base = binding.CTM(A, w.chi)
    base.ctm_step(2)
    C0, T0, Q0 = base.ctm_get_env()
    vals = []
    for sgn in (1.0, -1.0):
        c = binding.CTM(A + sgn * 1e-6 * V, w.chi)
        c.ctm_set_env(C0, T0, Q0)
        c.ctm_step(k)
        vals.append(c.ctm_energy(h)[1])
        c.close()
    fd = (vals[0] - vals[1]) / 2e-6
    assert abs(fd - np.sum(g * V)) <= 1e-5 * max(1.0, abs(fd))


def _zz_bonds():
    """S^z S^z on all three bonds.  On the converging near-product states every isotropic
    Kitaev-Heisenberg bond energy is stationary (K|S|^2 + 3J|S|^2 with |S| = 1/2 for
    any product state), so their gradients are tiny; this observable's are O(1)."""
    Sz = np.diag([0.5, -0.5])
    hz = np.kron(Sz, Sz)
    return np.stack([hz, hz, hz])


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_adjoint_k30_matches_cpu_reference(ctm_lib, precision):
    """k = 30 tracked steps (D = 4, chi = 32, converging near-product state) with the
    forward in the context's precision (split: BF16 slice contractions, FP64 QR) against
    the PyTorch float64 reference gradient through the same 30 steps."""
    import torch_reference as TR
    w = I.WORKLOADS["kitaev_D4_chi32_conv"]
    A, h = w.site_tensor(), _zz_bonds()
    E_gpu, g_gpu = _gpu_grad(A, w.chi, h, 3, 30, precision)
    env = _oracle_env_after(A, w.chi, 3)
    E_ref, g_ref = TR.energy_and_grad(A, env, h, 30)
    assert abs(E_gpu - E_ref) <= 1e-10
    assert np.max(np.abs(g_gpu - g_ref)) <= 1e-7 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("name,k", [("kitaev_D4_chi32_conv", 30), ("heis_D2_chi8", 10)])
def test_adjoint_tf32_forward(ctm_lib, name, k):
    """The FP32/TF32 forward with the FP64 QR: k tracked steps whose contractions are split-TF32
    products (about FP32 accuracy: (3 2^-21 + K 2^-23) relative, ~7e-5 at K = n = 512), the
    adjoint in FP64 from their checkpoints, against the float64 reference gradient through the
    same steps.  The forward's error carries into the energy and the gradient at most at that
    level (the near-product state hides most of it: its errors fall in the dominant direction
    that the normalisations remove; the random heis_D2_chi8 state shows it)."""
    import torch_reference as TR
    w = I.WORKLOADS[name]
    A, h = w.site_tensor(), _zz_bonds()
    E_gpu, g_gpu = _gpu_grad(A, w.chi, h, 3, k, "split_tf32")
    env = _oracle_env_after(A, w.chi, 3)
    E_ref, g_ref = TR.energy_and_grad(A, env, h, k)
    print(name, "tf32 forward: dE", abs(E_gpu - E_ref), "dg", np.max(np.abs(g_gpu - g_ref)) / np.max(np.abs(g_ref)))
    assert abs(E_gpu - E_ref) <= 1e-6                                   # measured 4e-9 (heis), 1e-13
    assert np.max(np.abs(g_gpu - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))   # measured 2e-8, 5e-11


def test_adjoint_d8_chi128_k30_split_forward(ctm_lib):
    """D = 8, chi = 128 (enlarged corner 8192 x 8192), converging near-product state: 3
    warm-up and 30 checkpointed steps in split-BF16 with the FP64 QR, the adjoint in
    FP64, against central differences (h = 1e-6) of the FP64 GPU forward through the
    same 30 steps from the same environment, along 3 random directions."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["kh_D8_chi128_conv"]
    A, h = w.site_tensor(), _zz_bonds()
    E, g = _gpu_grad(A, w.chi, h, 3, 30, "split_bf16")
    assert np.all(np.isfinite(g))
    base = binding.CTM(A, w.chi, precision="split_bf16", n_split=5)
    base.ctm_step(3)
    C0, T0, Q0 = base.ctm_get_env()
    base.close()
    rng = np.random.default_rng(8)
    for _ in range(3):
        V = rng.standard_normal(A.shape)
        vals = []
        for sgn in (1.0, -1.0):
            c = binding.CTM(A + sgn * 1e-6 * V, w.chi)
            c.ctm_set_env(C0, T0, Q0)
            c.ctm_step(30)
            vals.append(c.ctm_energy(h)[1])
            c.close()
        fd = (vals[0] - vals[1]) / 2e-6
        assert abs(fd - np.sum(g * V)) <= 1e-6 * max(1.0, abs(fd)), (fd, np.sum(g * V))


def test_autograd_reuses_context_and_defers_adjoint(ctm_lib):
    """Two differentiable energies of different tensors share one library context (the
    second starts from the first one's environment); a forward without backward runs no
    adjoint; each gradient matches a fresh ctm_grad from the environment it started at."""
    import torch
    from paper_2509_05090_gb300 import autograd as AG
    from paper_2509_05090_gb300 import binding
    AG.release_contexts()
    w = I.WORKLOADS["heis_D2_chi8"]
    h = torch.from_numpy(w.hamiltonians()).cuda()
    A1 = torch.from_numpy(w.site_tensor()).cuda().requires_grad_(True)
    E1 = AG.ctm_energy(A1, w.chi, h, warmup=5, k_tracked=3)
    (g1,) = torch.autograd.grad(E1, A1)
    assert len(AG._CONTEXTS) == 1
    ctm = next(iter(AG._CONTEXTS.values()))
    env1 = [x.clone() for x in ctm.ctm_get_env()]
    A2 = (A1.detach() * 1.01 + 0.001).requires_grad_(True)
    l0 = binding.ctm_kernel_launches()
    E2 = AG.ctm_energy(A2, w.chi, h, warmup=5, k_tracked=3)
    l_fwd = binding.ctm_kernel_launches() - l0
    (g2,) = torch.autograd.grad(E2, A2)
    l_bwd = binding.ctm_kernel_launches() - l0 - l_fwd
    # backward repeats the forward's steps and adds the adjoint (dozens of launches per
    # tracked step); the forward ran none of it
    assert l_bwd > l_fwd + 50, (l_fwd, l_bwd)
    assert len(AG._CONTEXTS) == 1 and next(iter(AG._CONTEXTS.values())) is ctm
    ref = binding.CTM(A2.detach(), w.chi)
    ref.ctm_set_env(*env1)
    E2r, g2r = ref.ctm_grad(h.cpu().numpy(), warmup=5, k_tracked=3)
    ref.close()
    assert abs(float(E2.detach()) - E2r) <= 1e-12
    assert torch.max(torch.abs(g2 - g2r)).item() <= 1e-10 * torch.max(torch.abs(g2r)).item()
    AG.release_contexts()


def test_lbfgs_optimisation_lowers_the_heisenberg_energy(ctm_lib):
    """Sec. II.D: L-BFGS over A with the adjoint gradient.  Heisenberg model with the
    pi-rotation on sublattice B (uniform ansatz), D = 2, chi = 16, from a seeded random
    tensor: the energy decreases at every iteration (strong-Wolfe line search), ends
    well below its start, and stays above the QMC ground-state energy -0.544553(20)
    (Sec. III.B) -- a variational upper bound."""
    from paper_2509_05090_gb300 import autograd as AG
    from paper_2509_05090_gb300.optimize import optimize
    AG.release_contexts()
    h = I.bond_hamiltonians(0.0, 1.0, rotate_b=True)
    A0 = I.random_site_tensor(2, 2, 2024)
    A, Es = optimize(A0, 16, h, steps=12, warmup=10, k_tracked=8)
    AG.release_contexts()
    assert all(b <= a + 1e-12 for a, b in zip(Es, Es[1:]))
    assert Es[-1] < Es[0] - 5e-3
    assert Es[-1] > -0.54457
    assert all(np.isfinite(Es))


def test_padded_warm_start_keeps_the_energy(ctm_lib):
    """A D = 2 tensor padded to D = 3 with a 1e-3 perturbation (Sec. II.D) gives a
    converged energy within the perturbation's effect of the D = 2 energy."""
    from paper_2509_05090_gb300 import binding
    from paper_2509_05090_gb300.optimize import pad_site_tensor
    h = I.bond_hamiltonians(0.0, 1.0, rotate_b=True)
    A2 = I.random_site_tensor(2, 2, 7)
    A3 = pad_site_tensor(A2, 3, 1e-3, 11)
    assert np.array_equal(A3[:, :2, :2, :2], A2)
    E = []
    for A, chi in ((A2, 16), (A3, 16)):
        c = binding.CTM(A, chi)
        c.ctm_converge(max_steps=300, tol=1e-11)
        E.append(c.ctm_energy(h)[1])
        c.close()
    assert abs(E[1] - E[0]) < 1e-3
