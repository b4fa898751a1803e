"""Thin ctypes binding of libctm (include/ctm.h), same names as the C ABI.

Argument marshalling only: every step of the CTMRG path runs in the CUDA
kernels of libctm.so.  PyTorch provides device memory (the workspace and the
input/output tensors) and the CUDA stream.  There is no CPU fallback: if the
library is missing or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ctm.h")

CTM_OK = 0
CTM_ENOTCONVERGED = 4
CTM_FP64 = 0
CTM_SPLIT_BF16 = 1
CTM_SPLIT_TF32 = 2
CTM_FP32_TF32 = 3
PRECISIONS = {"fp64": CTM_FP64, "split_bf16": CTM_SPLIT_BF16, "split_tf32": CTM_SPLIT_TF32, "fp32_tf32": CTM_FP32_TF32}


class ctm_config(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("D", ctypes.c_int), ("chi", ctypes.c_int),
                ("precision", ctypes.c_int), ("n_split", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_steps", ctypes.c_int), ("symmetrize", ctypes.c_int), ("corner_mode", ctypes.c_int),
                ("deterministic", ctypes.c_int)]


class CtmError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_str(status)}")


_lib = None


def header_functions(path: str = HEADER):
    """Names of the functions include/ctm.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ctm_[a-z_0-9]+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    """Load libctm.so (built in-tree by build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libctm.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    I = ctypes.c_int
    cfgp = ctypes.POINTER(ctm_config)
    sigs = {
        "ctm_workspace_bytes": (ctypes.c_size_t, [cfgp]),
        "ctm_init": (I, [cfgp, P, P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
        "ctm_step": (I, [P, I, dp]),
        "ctm_converge": (I, [P, I, ctypes.c_double, I, ctypes.POINTER(I), dp]),
        "ctm_energy": (I, [P, P, dp, dp, dp]),
        "ctm_get_env": (I, [P, P, P, P]),
        "ctm_set_env": (I, [P, P, P, P]),
        "ctm_get_intermediate": (I, [P, I, P, ctypes.c_size_t]),
        "ctm_destroy": (None, [P]),
        "ctm_status_str": (ctypes.c_char_p, [I]),
        "ctm_version": (ctypes.c_char_p, []),
        "ctm_step_profiled": (I, [P, dp, I]),
        "ctm_kernel_launches": (ctypes.c_ulonglong, []),
        "ctm_gemm_workspace_bytes": (ctypes.c_size_t, [I, I, I, I, I]),
        "ctm_gemm": (I, [I, I, I, P, P, P, I, I, P, ctypes.c_size_t, P]),
        "ctm_gemm_noalloc": (I, [I, I, I, P, P, P, I, I, P]),
        "ctm_grad_workspace_bytes": (ctypes.c_size_t, [P, I]),
        "ctm_batch_workspace_bytes": (ctypes.c_size_t, [P, I]),
        "ctm_batch_init": (I, [P, I, P, P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
        "ctm_batch_step": (I, [P, I, dp]),
        "ctm_batch_ctx": (I, [P, I, ctypes.POINTER(P)]),
        "ctm_batch_destroy": (None, [P]),
        "ctm_grad": (I, [P, I, I, P, P, ctypes.c_size_t, dp, P]),
        "ctm_debug_force_timeout": (I, [P, I]),
        "ctm_probe_fp64_peak": (I, [P, dp]),
        "ctm_set_site": (I, [P, P, I]),
        "ctm_complex_workspace_bytes": (ctypes.c_size_t, [cfgp, I]),
        "ctm_complex_init": (I, [cfgp, I, P, P, ctypes.c_size_t, P, ctypes.POINTER(P)]),
        "ctm_complex_step": (I, [P, I, dp]),
        "ctm_complex_converge": (I, [P, I, ctypes.c_double, I, ctypes.POINTER(I), dp]),
        "ctm_complex_energy": (I, [P, P, dp, dp, dp]),
        "ctm_complex_get_env": (I, [P, P, P, P]),
        "ctm_complex_set_env": (I, [P, P, P, P]),
        "ctm_complex_get_intermediate": (I, [P, I, P, ctypes.c_size_t]),
        "ctm_complex_destroy": (None, [P]),
        "ctm_transfer_workspace_bytes": (ctypes.c_size_t, [P, I]),
        "ctm_transfer_spectrum": (I, [P, I, I, ctypes.c_double, P, ctypes.c_size_t, dp, dp, dp,
                                      ctypes.POINTER(I)]),
        "ctm_complex_transfer_workspace_bytes": (ctypes.c_size_t, [P, I]),
        "ctm_complex_transfer_spectrum": (I, [P, I, I, ctypes.c_double, P, ctypes.c_size_t, dp, dp, dp,
                                              ctypes.POINTER(I)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def ctm_kernel_launches() -> int:
    return int(load().ctm_kernel_launches())


def ctm_probe_fp64_peak() -> float:
    """Measured FP64 (DFMA) peak of the current device in TFLOP/s."""
    torch = _torch()
    t = ctypes.c_double(0.0)
    st = load().ctm_probe_fp64_peak(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(t))
    if st != CTM_OK:
        raise CtmError(st, "ctm_probe_fp64_peak")
    return t.value


def ctm_gemm(A, B, precision="fp64", n_split=4):
    """C = A B through the library's contraction engine (torch CUDA float64 tensors)."""
    torch = _torch()
    A = A.to(device="cuda", dtype=torch.float64).contiguous()
    B = B.to(device="cuda", dtype=torch.float64).contiguous()
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    nbytes = int(load().ctm_gemm_workspace_bytes(M, N, K, prec, n_split))
    if nbytes == 0:
        raise CtmError(1, "ctm_gemm_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    st = load().ctm_gemm(M, N, K, _ptr(A), _ptr(B), _ptr(C), prec, int(n_split), _ptr(ws), nbytes,
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != CTM_OK:
        raise CtmError(st, "ctm_gemm")
    return C


def ctm_gemm_noalloc(A, B, precision="fp64", n_split=4):
    """C = A B through ctm_gemm_noalloc: no workspace, the library's fixed device scratch."""
    torch = _torch()
    A = A.to(device="cuda", dtype=torch.float64).contiguous()
    B = B.to(device="cuda", dtype=torch.float64).contiguous()
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    st = load().ctm_gemm_noalloc(M, N, K, _ptr(A), _ptr(B), _ptr(C), prec, int(n_split),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != CTM_OK:
        raise CtmError(st, "ctm_gemm_noalloc")
    return C


def status_str(status: int) -> str:
    return load().ctm_status_str(int(status)).decode()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libctm needs a CUDA device; there is no CPU fallback")
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


CORNER_MODES = {"qmq": 0, "r": 1}


def make_config(d, D, chi, precision="fp64", n_split=3, tol=1e-10, max_steps=200, symmetrize=True, corner="qmq",
                deterministic=False):
    return ctm_config(int(d), int(D), int(chi), PRECISIONS[precision] if isinstance(precision, str) else
                      int(precision), int(n_split), float(tol), int(max_steps), 1 if symmetrize else 0,
                      CORNER_MODES[corner], 1 if deterministic else 0)


def ctm_workspace_bytes(cfg: ctm_config) -> int:
    return int(load().ctm_workspace_bytes(ctypes.byref(cfg)))


class CTM:
    """One CTMRG instance on the current CUDA device (ctm_init ... ctm_destroy)."""

    def __init__(self, A, chi, precision="fp64", n_split=3, tol=1e-10, max_steps=200, symmetrize=True,
                 stream=None, corner="qmq", deterministic=False):
        torch = _torch()
        lib = load()
        if isinstance(A, np.ndarray):
            A = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64)).cuda()
        A = A.to(device="cuda", dtype=torch.float64).contiguous()
        d, D = int(A.shape[0]), int(A.shape[1])
        self.d, self.D, self.chi = d, D, int(chi)
        self.D2 = D * D
        self.n = self.chi * self.D2
        self.cfg = make_config(d, D, chi, precision, n_split, tol, max_steps, symmetrize, corner, deterministic)
        nbytes = ctm_workspace_bytes(self.cfg)
        if nbytes == 0:
            raise CtmError(1, "ctm_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self._A = A
        h = ctypes.c_void_p()
        st = lib.ctm_init(ctypes.byref(self.cfg), _ptr(A), _ptr(self.workspace), nbytes,
                          ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != CTM_OK:
            raise CtmError(st, "ctm_init")
        self._h = h

    # --- calls ---------------------------------------------------------
    def ctm_step(self, nsteps=1, want_delta=True):
        d = ctypes.c_double(float("nan"))
        st = load().ctm_step(self._h, int(nsteps), ctypes.byref(d) if want_delta else None)
        if st != CTM_OK:
            raise CtmError(st, "ctm_step")
        return d.value if want_delta else None

    def ctm_converge(self, max_steps=0, tol=0.0, check_every=1, raise_not_converged=False):
        steps = ctypes.c_int(0)
        delta = ctypes.c_double(float("nan"))
        st = load().ctm_converge(self._h, int(max_steps), float(tol), int(check_every), ctypes.byref(steps),
                                 ctypes.byref(delta))
        if st not in (CTM_OK, CTM_ENOTCONVERGED) or (st != CTM_OK and raise_not_converged):
            raise CtmError(st, "ctm_converge")
        return steps.value, delta.value, st == CTM_OK

    def ctm_energy(self, h):
        torch = _torch()
        if isinstance(h, np.ndarray):
            h = torch.from_numpy(np.ascontiguousarray(h, dtype=np.float64))
        h = h.to(device="cuda", dtype=torch.float64).contiguous()
        dd = self.d * self.d
        e = (ctypes.c_double * 3)()
        es = ctypes.c_double()
        rho = (ctypes.c_double * (dd * dd))()
        st = load().ctm_energy(self._h, _ptr(h), e, ctypes.byref(es), rho)
        if st != CTM_OK:
            raise CtmError(st, "ctm_energy")
        return np.array(e[:]), es.value, np.array(rho[:]).reshape(dd, dd)

    def ctm_grad(self, h, warmup=10, k_tracked=24):
        """(E_site, dE/dA) by the hand-written adjoint; dA has the layout of the raw A given to ctm_init."""
        torch = _torch()
        if isinstance(h, np.ndarray):
            h = torch.from_numpy(np.ascontiguousarray(h, dtype=np.float64))
        h = h.to(device="cuda", dtype=torch.float64).contiguous()
        nbytes = int(load().ctm_grad_workspace_bytes(self._h, int(k_tracked)))
        if nbytes == 0:
            raise CtmError(1, "ctm_grad_workspace_bytes")
        gws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        dA = torch.empty_like(self._A)
        E = ctypes.c_double()
        st = load().ctm_grad(self._h, int(warmup), int(k_tracked), _ptr(h), _ptr(gws), nbytes, ctypes.byref(E),
                             _ptr(dA))
        if st != CTM_OK:
            raise CtmError(st, "ctm_grad")
        return E.value, dA

    def ctm_transfer_spectrum(self, nev=3, max_iter=2000, tol=1e-12):
        """(lambda[0..nev) normalised magnitudes, xi, ln(lambda_1/lambda_2), iterations, converged)."""
        torch = _torch()
        nbytes = int(load().ctm_transfer_workspace_bytes(self._h, int(nev)))
        if nbytes == 0:
            raise CtmError(1, "ctm_transfer_workspace_bytes")
        tws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        lam = (ctypes.c_double * nev)()
        xi, gap, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        st = load().ctm_transfer_spectrum(self._h, int(nev), int(max_iter), float(tol), _ptr(tws), nbytes, lam,
                                          ctypes.byref(xi), ctypes.byref(gap), ctypes.byref(it))
        if st not in (CTM_OK, CTM_ENOTCONVERGED):
            raise CtmError(st, "ctm_transfer_spectrum")
        return np.array(lam[:]), xi.value, gap.value, it.value, st == CTM_OK

    def ctm_set_site(self, A, reset_env=False):
        """Replace the site tensor (same d, D); keep (or reset) the environment."""
        torch = _torch()
        if isinstance(A, np.ndarray):
            A = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64))
        A = A.to(device="cuda", dtype=torch.float64).contiguous()
        if tuple(A.shape) != (self.d, self.D, self.D, self.D):
            raise CtmError(1, "ctm_set_site")
        st = load().ctm_set_site(self._h, _ptr(A), 1 if reset_env else 0)
        if st != CTM_OK:
            raise CtmError(st, "ctm_set_site")
        self._A = A

    def ctm_get_env(self):
        torch = _torch()
        C = torch.empty((self.chi, self.chi), dtype=torch.float64, device="cuda")
        T = torch.empty((self.chi, self.D2, self.chi), dtype=torch.float64, device="cuda")
        Q = torch.empty((self.n, self.chi), dtype=torch.float64, device="cuda")
        st = load().ctm_get_env(self._h, _ptr(C), _ptr(T), _ptr(Q))
        if st != CTM_OK:
            raise CtmError(st, "ctm_get_env")
        return C, T, Q

    def ctm_set_env(self, C, T, Q):
        torch = _torch()
        conv = [(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)) if isinstance(x, np.ndarray) else x)
                .to(device="cuda", dtype=torch.float64).contiguous() for x in (C, T, Q)]
        st = load().ctm_set_env(self._h, *[_ptr(x) for x in conv])
        if st != CTM_OK:
            raise CtmError(st, "ctm_set_env")

    _SHAPES = {0: "M", 1: "Y", 2: "R", 3: "Q", 4: "s", 5: "A", 6: "a"}

    def ctm_get_intermediate(self, which):
        torch = _torch()
        if isinstance(which, str):
            which = {v: k for k, v in self._SHAPES.items()}[which]
        n, chi, D2 = self.n, self.chi, self.D2
        shape = {0: (n, n), 1: (n, chi), 2: (chi, chi), 3: (n, chi), 4: (chi,),
                 5: (self.d, self.D, self.D, self.D), 6: (D2, D2, D2)}[which]
        out = torch.empty(shape, dtype=torch.float64, device="cuda")
        st = load().ctm_get_intermediate(self._h, int(which), _ptr(out), out.numel())
        if st != CTM_OK:
            raise CtmError(st, "ctm_get_intermediate")
        return out

    PHASES = ("enlarged_corner", "reduced_corner", "qr", "corner", "edge", "spectrum_wait", "handover")
    SIDE_PHASES = ("spectrum", "gemm_kernels", "prepass")

    def ctm_step_profiled(self):
        ms = (ctypes.c_double * 10)()
        st = load().ctm_step_profiled(self._h, ms, 10)
        if st != CTM_OK:
            raise CtmError(st, "ctm_step_profiled")
        out = dict(zip(self.PHASES, ms[:7]))
        out["spectrum"] = ms[7]       # side stream, overlaps the next step in ctm_step
        out["gemm_kernels"] = ms[8]   # the contraction-engine kernels alone (subset of the phases)
        out["prepass"] = ms[9]        # the split engine's operand pre-pass (subset of the phases)
        return out

    def ctm_debug_force_timeout(self, enable=True):
        st = load().ctm_debug_force_timeout(self._h, 1 if enable else 0)
        if st != CTM_OK:
            raise CtmError(st, "ctm_debug_force_timeout")

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            load().ctm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


IRREPS = {"A1": 0, "E": 1}


def _complex_dev(x, torch):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128))
    return x.to(device="cuda", dtype=torch.complex128).contiguous()


class CTMComplex:
    """One complex (E- or A1-irrep) CTMRG instance (ctm_complex_init ... ctm_complex_destroy).
    Complex tensors go in and out as torch.complex128 on the current CUDA device."""

    def __init__(self, A, chi, irrep="E", precision="fp64", n_split=5, tol=1e-10, max_steps=200, symmetrize=True,
                 stream=None, deterministic=False, corner="qmq"):
        torch = _torch()
        lib = load()
        A = _complex_dev(A, torch)
        if A.dim() != 4 or not (A.shape[1] == A.shape[2] == A.shape[3]):
            raise ValueError(f"site tensor must be d x D x D x D, got {tuple(A.shape)}")
        d, D = int(A.shape[0]), int(A.shape[1])
        self.d, self.D, self.chi = d, D, int(chi)
        self.D2 = D * D
        self.n = self.chi * self.D2
        self.irrep = IRREPS[irrep] if isinstance(irrep, str) else int(irrep)
        self.cfg = make_config(d, D, chi, precision, n_split, tol, max_steps, symmetrize, corner, deterministic)
        nbytes = int(lib.ctm_complex_workspace_bytes(ctypes.byref(self.cfg), self.irrep))
        if nbytes == 0:
            raise CtmError(1, "ctm_complex_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self._A = A
        h = ctypes.c_void_p()
        st = lib.ctm_complex_init(ctypes.byref(self.cfg), self.irrep, _ptr(A), _ptr(self.workspace), nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != CTM_OK:
            raise CtmError(st, "ctm_complex_init")
        self._h = h

    def ctm_complex_step(self, nsteps=1, want_delta=True):
        d = ctypes.c_double(float("nan"))
        st = load().ctm_complex_step(self._h, int(nsteps), ctypes.byref(d) if want_delta else None)
        if st != CTM_OK:
            raise CtmError(st, "ctm_complex_step")
        return d.value if want_delta else None

    def ctm_complex_converge(self, max_steps=0, tol=0.0, check_every=1):
        steps = ctypes.c_int(0)
        delta = ctypes.c_double(float("nan"))
        st = load().ctm_complex_converge(self._h, int(max_steps), float(tol), int(check_every), ctypes.byref(steps),
                                         ctypes.byref(delta))
        if st not in (CTM_OK, CTM_ENOTCONVERGED):
            raise CtmError(st, "ctm_complex_converge")
        return steps.value, delta.value, st == CTM_OK

    def ctm_complex_energy(self, h):
        """h: three d^2 x d^2 complex bond operators (x, y, z); returns (e_bond, E_site, rho_z)."""
        torch = _torch()
        h = _complex_dev(h, torch)
        dd = self.d * self.d
        if h.numel() != 3 * dd * dd:
            raise ValueError(f"need three {dd} x {dd} bond operators, got {tuple(h.shape)}")
        e = (ctypes.c_double * 3)()
        es = ctypes.c_double()
        rho = (ctypes.c_double * (2 * dd * dd))()
        st = load().ctm_complex_energy(self._h, _ptr(h), e, ctypes.byref(es), rho)
        if st != CTM_OK:
            raise CtmError(st, "ctm_complex_energy")
        r = np.array(rho[:])
        return np.array(e[:]), es.value, (r[0::2] + 1j * r[1::2]).reshape(dd, dd)

    def ctm_complex_transfer_spectrum(self, nev=3, max_iter=2000, tol=1e-12):
        """(lambda[0..nev) normalised magnitudes, xi, ln(lambda_1/lambda_2), iterations, converged)
        of the complex environment's column transfer matrix."""
        torch = _torch()
        nbytes = int(load().ctm_complex_transfer_workspace_bytes(self._h, int(nev)))
        if nbytes == 0:
            raise CtmError(1, "ctm_complex_transfer_workspace_bytes")
        tws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        lam = (ctypes.c_double * nev)()
        xi, gap, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        st = load().ctm_complex_transfer_spectrum(self._h, int(nev), int(max_iter), float(tol), _ptr(tws), nbytes,
                                                  lam, ctypes.byref(xi), ctypes.byref(gap), ctypes.byref(it))
        if st not in (CTM_OK, CTM_ENOTCONVERGED):
            raise CtmError(st, "ctm_complex_transfer_spectrum")
        return np.array(lam[:]), xi.value, gap.value, it.value, st == CTM_OK

    def ctm_complex_get_env(self):
        torch = _torch()
        C = torch.empty((self.chi, self.chi), dtype=torch.complex128, device="cuda")
        T = torch.empty((self.chi, self.D2, self.chi), dtype=torch.complex128, device="cuda")
        Q = torch.empty((self.n, self.chi), dtype=torch.complex128, device="cuda")
        st = load().ctm_complex_get_env(self._h, _ptr(C), _ptr(T), _ptr(Q))
        if st != CTM_OK:
            raise CtmError(st, "ctm_complex_get_env")
        return C, T, Q

    def ctm_complex_set_env(self, C, T, Q):
        torch = _torch()
        conv = [_complex_dev(x, torch) for x in (C, T, Q)]
        for x, cnt, name in zip(conv, (self.chi ** 2, self.chi * self.D2 * self.chi, self.n * self.chi), "CTQ"):
            if x.numel() != cnt:
                raise ValueError(f"{name} has {x.numel()} elements, expected {cnt}")
        st = load().ctm_complex_set_env(self._h, *[_ptr(x) for x in conv])
        if st != CTM_OK:
            raise CtmError(st, "ctm_complex_set_env")

    _SHAPES = {0: "M", 1: "Y", 2: "R", 3: "Q", 4: "s", 5: "A", 6: "a", 7: "C", 8: "T"}

    def ctm_complex_get_intermediate(self, which):
        torch = _torch()
        if isinstance(which, str):
            which = {v: k for k, v in self._SHAPES.items()}[which]
        n, chi, D2, D = self.n, self.chi, self.D2, self.D
        shape = {0: (n, n), 1: (n, chi), 2: (chi, chi), 3: (n, chi), 4: (chi,), 5: (self.d, D, D, D),
                 6: (D2, D2, D2), 7: (chi, chi), 8: (chi, D2, chi)}[which]
        out = torch.empty(shape, dtype=torch.float64 if which == 4 else torch.complex128, device="cuda")
        count = out.numel() * (1 if which == 4 else 2)
        st = load().ctm_complex_get_intermediate(self._h, int(which), _ptr(out), count)
        if st != CTM_OK:
            raise CtmError(st, "ctm_complex_get_intermediate")
        return out

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            load().ctm_complex_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _CtxView(CTM):
    """A context owned by a batch (no workspace of its own; not destroyed here)."""

    def __init__(self, handle, d, D, chi, A, stream):
        self._h = handle
        self.d, self.D, self.chi = d, D, chi
        self.D2 = D * D
        self.n = chi * self.D2
        self._A = A
        self.stream = stream

    def close(self):
        self._h = None


class CTMBatch:
    """Ragged batch of instances advanced together (ctm_batch_* of include/ctm.h)."""

    def __init__(self, tensors, chis, precision="split_bf16", n_split=5, tol=1e-10, max_steps=200, stream=None):
        torch = _torch()
        lib = load()
        As = []
        for A in tensors:
            if isinstance(A, np.ndarray):
                A = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64))
            As.append(A.to(device="cuda", dtype=torch.float64).contiguous())
        self._A = As
        cfgs = (ctm_config * len(As))(*[make_config(A.shape[0], A.shape[1], chi, precision, n_split, tol, max_steps)
                                        for A, chi in zip(As, chis)])
        self._cfgs = cfgs
        self.chis = [int(c) for c in chis]
        nbytes = int(lib.ctm_batch_workspace_bytes(ctypes.cast(cfgs, ctypes.c_void_p), len(As)))
        if nbytes == 0:
            raise CtmError(1, "ctm_batch_workspace_bytes")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        ptrs = (ctypes.c_void_p * len(As))(*[A.data_ptr() for A in As])
        h = ctypes.c_void_p()
        st = lib.ctm_batch_init(ctypes.cast(cfgs, ctypes.c_void_p), len(As), ctypes.cast(ptrs, ctypes.c_void_p),
                                _ptr(self.workspace), nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                ctypes.byref(h))
        if st != CTM_OK:
            raise CtmError(st, "ctm_batch_init")
        self._h = h

    def ctm_batch_step(self, nsteps=1, want_delta=False):
        d = ctypes.c_double(float("nan"))
        st = load().ctm_batch_step(self._h, int(nsteps), ctypes.byref(d) if want_delta else None)
        if st != CTM_OK:
            raise CtmError(st, "ctm_batch_step")
        return d.value if want_delta else None

    def instance(self, i):
        h = ctypes.c_void_p()
        st = load().ctm_batch_ctx(self._h, int(i), ctypes.byref(h))
        if st != CTM_OK:
            raise CtmError(st, "ctm_batch_ctx")
        A = self._A[i]
        return _CtxView(h, int(A.shape[0]), int(A.shape[1]), self.chis[i], A, self.stream)

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            load().ctm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
