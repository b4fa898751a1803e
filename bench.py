#!/usr/bin/env python
"""Benchmark: QR-based C3v CTMRG steps/s on one GB300 (replicas across GPUs).

Default workload: d = 2, D = 6, chi = 72 (enlarged corner 2592 x 2592),
Kitaev-Heisenberg phi = 0.3 pi, seeded random C3v-projected site tensor.
A "step" is one full CTMRG renormalisation step (enlarged corner, reduced
corner, Householder QR, corner and edge renormalisation, corner spectrum and
delta).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|split_bf16]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CTMRG steps/s & time-to-converged env at D=6,χ=72; mixed vs FP64 at ≤1e-9 dE"
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes of the step's 11 contraction launches, from one ncu capture per
# workload (--metrics dram__bytes_read.sum,dram__bytes_write.sum on the launches
# of one step, plans replayed from the plain run's autotune cache).  Set back to
# absent whenever the contraction kernel changes.
NCU_TRAFFIC = {("kh_D6_chi72", "split_bf16", 5): 400.4e6}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def step_gemm_flops(chi, D2):
    """Algorithmic FP64 flops of the GEMM phases of one step (2 x MACs)."""
    n = chi * D2
    macs = [
        n * chi * chi,            # W = T C
        n * n * chi,              # X = W T^T
        chi * chi * D2 * D2 * D2,  # Y1 = X a
        chi * chi * D2 * D2 * D2,  # M = Y1 a
        n * chi * n,              # Y = M Qs
        n * chi * n,              # M Q
        chi * chi * n,            # Q^T (M Q)
        n * n * chi,              # H1 = T Q
        chi * chi * D2 * D2 * D2,  # H2
        chi * chi * D2 * D2 * D2,  # H3
        chi * n * n,              # T' = Q^T H3
    ]
    return 2.0 * sum(macs)


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled about every millisecond while
    the timed region runs, read through NVML (the driver's libnvidia-ml, via ctypes);
    nvidia-smi polling (100 ms) if NVML cannot be opened."""

    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []      # (sm_mhz, reason bits)
        self.max_mhz = None
        self.source = None
        self._stop = threading.Event()
        self.proc = None
        self.lines = []

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(self.gpu).uuid)
        except Exception:
            uuid = None
        if not uuid or lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) != 0:
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return lib, h, reasons

    def _nvml_loop(self, lib, h, reasons):
        import ctypes
        mhz, mx, bits = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
            self.max_mhz = float(mx.value)
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and reasons(h, ctypes.byref(bits)) == 0:
                self.samples.append((float(mhz.value), int(bits.value)))
            time.sleep(0.0005)

    def __enter__(self):
        try:
            lib, h, reasons = self._nvml_handle()
            self.source = "nvml ~1 ms"
            self.t = threading.Thread(target=self._nvml_loop, args=(lib, h, reasons), daemon=True)
            self.t.start()
            time.sleep(0.003)   # first samples before the timed work starts
            return self
        except Exception:
            pass
        try:
            self.source = "nvidia-smi 100 ms"
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        elif getattr(self, "t", None):
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        if self.samples:
            for mhz, bits in self.samples:
                sm.append(mhz)
                for b, nm in self.REASONS.items():
                    if bits & b:
                        reasons.add(nm)
            mx = [self.max_mhz] if self.max_mhz else [max(sm)]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": self.source}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, ws, device="cuda"):
    """Each value's maximum over the ranks of the process group (the replicas' timings:
    the job is as slow as its slowest rank); identity for one rank."""
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_throughput(total_ms_max, steps, ws):
    """Whole-job steps/s of ws independent replicas that each ran `steps` steps, timed by
    the slowest rank's total_ms_max; and the ms per step."""
    return ws * steps / (total_ms_max / 1e3), total_ms_max / steps


def cpu_oracle_rate(w, budget_s=20.0, max_steps=None, threads=1, warmup=0):
    """The FP64 CPU oracle as it stands on bounded steps of the workload, after `warmup`
    untimed steps; threads = 0: all cores (its loops are OpenMP-parallel over output rows).
    Returns (steps/s, steps, seconds, init seconds, threads used)."""
    from oracle import oracle as orc
    used = orc.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    A = w.site_tensor()
    t0 = time.perf_counter()
    ctm = orc.OracleCTM(A, w.chi)
    init_s = time.perf_counter() - t0
    for _ in range(warmup):
        ctm.step()
    times = []
    while True:
        t = time.perf_counter()
        ctm.step()
        times.append(time.perf_counter() - t)
        if sum(times) >= budget_s or (max_steps and len(times) >= max_steps):
            break
    return len(times) / sum(times), len(times), sum(times), init_s, used


def run_reference(args, w):
    ws, rank, local = dist_setup()
    if rank != 0:
        return 0
    budget = min(150.0, max(10.0, 8.0 * args.steps))
    # W untimed warm-up steps, then K timed steps (fewer if the time budget runs out first)
    rate, nsteps, secs, _, used = cpu_oracle_rate(w, budget_s=budget, max_steps=args.steps, threads=0,
                                                  warmup=args.warmup)
    line = {
        "metric": METRIC, "value": rate, "unit": "steps/s", "n_gpus": args.gpus, "steps": nsteps,
        "warmup": args.warmup, "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "d": w.d, "D": w.D, "chi": w.chi, "n": w.n, "precision": "fp64"},
        "impl": "reference",
        "cpu_baseline": {"value": rate, "unit": "steps/s", "cores": used, "host_cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": f"{nsteps} plain-C FP64 oracle steps of {w.name} after {args.warmup} "
                                   f"untimed ones from the initial environment ({secs:.1f} s, {used} OpenMP "
                                   f"threads)"},
        "e2e": {"value": rate, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_record(args, steps):
    """96 independent Kitaev-Heisenberg instances (phi = 2 pi i / 96, D in 3..6, chi in 24..72):
    aggregate instance-steps/s of the batch (one graph launch per batched step, split-BF16
    contractions with autotuned tiles) against one-instance-at-a-time FP64 launches."""
    import torch
    from paper_2509_05090_gb300 import binding, inputs
    wl = inputs.batch_workload()
    tensors = [w.site_tensor() for w in wl]
    chis = [w.chi for w in wl]
    t_init = time.perf_counter()
    batch = binding.CTMBatch(tensors, chis, precision=args.precision, n_split=args.n_split)
    batch.ctm_batch_step(2)   # eager (autotuning) step, then the captured graph's first replay
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_init
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l_timed = binding.ctm_kernel_launches()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(batch.stream)
        batch.ctm_batch_step(steps)
        e1.record(batch.stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kernels_per_step = (binding.ctm_kernel_launches() - l_timed) // steps   # kernels of one replay
    value = len(wl) * steps / (ms / 1e3)
    flops = sum(step_gemm_flops(w.chi, w.D2) for w in wl)
    T = args.n_split
    pairs = T * (T + 1) // 2 if args.precision != "fp64" else 1
    peaks, src = _peaks()
    achieved = pairs * flops / (ms / steps / 1e3) / 1e12
    rec = {"value": value, "unit": "instance-steps/s", "instances": len(wl), "steps": steps,
           "ms_per_batched_step": ms / steps, "setup_s": setup_s,
           "kernels_per_batched_step": int(kernels_per_step),
           "launch": "one CUDA graph launch per batched step",
           "tensor_frac_of_bf16_burst": achieved / peaks["bf16_tflops"] if args.precision != "fp64" else None,
           "clocks": clk.summary()}
    batch.close()
    # baseline: the same instances in FP64, one instance at a time (its own launches, no batching)
    base_ms = 0.0
    for A, chi in zip(tensors, chis):
        c = binding.CTM(A, chi, precision="fp64")
        c.ctm_step(1, want_delta=False)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(c.stream)
        for _ in range(steps):   # one launch sequence per instance and step
            c.ctm_step(1, want_delta=False)
        b1.record(c.stream)
        torch.cuda.synchronize()
        base_ms += b0.elapsed_time(b1)
        c.close()
    rec["fp64_one_instance_at_a_time"] = {"value": len(wl) * steps / (base_ms / 1e3), "unit": "instance-steps/s"}
    return rec


def run_batch(args):
    """The ragged batch as the benchmark's own workload (--workload batch96)."""
    import torch
    from paper_2509_05090_gb300 import inputs
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        if rank != 0:
            return 0
        wl = inputs.batch_workload()
        t_tot, n_tot = 0.0, 0
        for w in wl[:: max(1, len(wl) // 4)]:
            r, n, secs, _, used = cpu_oracle_rate(w, budget_s=8.0, max_steps=2, threads=0)
            t_tot += secs
            n_tot += n
        rate = n_tot / t_tot
        print(json.dumps({"metric": METRIC + " [ragged batch of 96]", "value": rate, "unit": "instance-steps/s",
                          "n_gpus": args.gpus, "steps": n_tot, "warmup": 0, "ms_per_step": 1e3 / rate,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": "batch96"}, "impl": "reference",
                          "cpu_baseline": {"value": rate, "unit": "instance-steps/s", "cores": used, "kind": "oracle",
                                           "sample": f"{n_tot} oracle steps on 4 of the 96 instances"},
                          "e2e": {"value": rate, "unit": "instance-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    torch.cuda.set_device(local)
    rec = batch_record(args, args.steps)
    T = args.n_split
    line = {"metric": METRIC + " [ragged batch of 96]", "value": rec["value"], "unit": "instance-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_batched_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else f"bf16x{T}-split+f64",
            "data": "synthetic (seeded C3v-projected tensors, Kitaev-Heisenberg phi_i = 2 pi i/96)",
            "config": {"workload": "batch96", "instances": rec["instances"], "D": "3..6", "chi": "24..72",
                       "precision": args.precision, "launch": rec["launch"],
                       "l2": "batched step working set several GB > L2"},
            "clocks": rec["clocks"], "gpu_launches": rec["kernels_per_batched_step"] * args.steps,
            "batch96": rec}
    print(json.dumps(line), flush=True)
    return 0


def energy_vs_oracle(w, precision, n_split, steps):
    """Energy after `steps` steps from the initial environment on the GPU (precision) and in
    the oracle (all cores): (E_gpu, E_oracle)."""
    from oracle import oracle as orc
    from paper_2509_05090_gb300 import binding
    A, h = w.site_tensor(), w.hamiltonians()
    g = binding.CTM(A, w.chi, precision=precision, n_split=n_split)
    g.ctm_step(steps, want_delta=False)
    _, E, _ = g.ctm_energy(h)
    g.close()
    orc.set_threads(os.cpu_count() or 1)
    ref = orc.OracleCTM(A, w.chi)
    for _ in range(steps):
        ref.step()
    return E, ref.energy(h)[1]


def time_to_converged(w, precision, n_split, max_steps, corner="qmq", spectrum=False):
    """Wall time from ctm_init to a converged environment (delta < tol, read back every
    step) and the energy there."""
    import torch
    from paper_2509_05090_gb300 import binding
    A, h = w.site_tensor(), w.hamiltonians()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = binding.CTM(A, w.chi, precision=precision, n_split=n_split, corner=corner)
    nst, dl, ok = g.ctm_converge(max_steps=max_steps, tol=w.tol, check_every=1)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    _, E, _ = g.ctm_energy(h)
    rec = {"steps": nst, "delta": dl, "converged": ok, "seconds": secs, "E_site": E}
    if spectrum:
        # transfer-matrix spectrum of the converged environment (Sec. II.C, Eq. 3)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        # lambda_2, lambda_3 ~ 6e-6 lie in a cluster of near-equal magnitudes here, so the
        # ratios lambda_i / lambda_1 are asked stable to 1e-9 (not the default 1e-12)
        lam, xi, gap, iters, sok = g.ctm_transfer_spectrum(nev=3, max_iter=200, tol=1e-9)
        rec["transfer_spectrum"] = {"tol": 1e-9, "lambda": [float(x) for x in lam], "xi_bravais": xi,
                                    "ln_lambda1_over_lambda2": gap, "iterations": iters, "converged": sok,
                                    "seconds": time.perf_counter() - t1}
    g.close()
    return rec


def fp64_step_record(w, steps, fp64_peak):
    """FP64 steps of workload w (one captured graph of `steps` steps), CUDA-event timed."""
    import torch
    from paper_2509_05090_gb300 import binding
    c = binding.CTM(w.site_tensor(), w.chi, precision="fp64")
    c.ctm_step(1, want_delta=False)       # eager first step
    c.ctm_step(steps, want_delta=False)   # capture + run the K-step graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(c.stream)
    c.ctm_step(steps, want_delta=False)
    e1.record(c.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ph = {k: 0.0 for k in binding.CTM.PHASES + binding.CTM.SIDE_PHASES}
    for _ in range(2):
        for k, v in c.ctm_step_profiled().items():
            ph[k] += v / 2
    c.close()
    flops = step_gemm_flops(w.chi, w.D2)
    return {"workload": w.name, "steps_per_s": 1e3 / ms, "ms_per_step": ms,
            "contraction_tflops": flops / (ph["gemm_kernels"] / 1e3) / 1e12,
            "contraction_frac_of_fp64_peak": flops / (ph["gemm_kernels"] / 1e3) / 1e12 / fp64_peak,
            "step_tflops": flops / (ms / 1e3) / 1e12, "step_frac_of_fp64_peak": flops / (ms / 1e3) / 1e12 / fp64_peak,
            "fp64_peak_tflops": fp64_peak, "phase_ms": ph, "algorithmic_flops_per_step": flops}


def grad_record(fp64_peak, warmup=3, k_tracked=30):
    """The differentiation configuration: D = 8, chi = 128 (enlarged corner 8192 x 8192), the
    FP32/TF32 forward (split TF32 contractions, FP64 QR) over `warmup` + `k_tracked`
    checkpointed steps of the converging Kitaev-Heisenberg state, the energy, and the
    hand-written FP64 adjoint (ctm_grad).  The forward alone (same steps, energy) is timed on
    a second context so that the adjoint's share can be stated; the adjoint recomputes each
    tracked step in FP64 and runs two FP64 products per contraction, so its algorithmic work
    is 3 k_tracked step GEMMs."""
    import torch
    from paper_2509_05090_gb300 import binding, inputs
    w = inputs.WORKLOADS["kh_D8_chi128_conv"]
    A, h = w.site_tensor(), w.hamiltonians()
    c = binding.CTM(A, w.chi, precision="split_tf32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E, dA = c.ctm_grad(h, warmup=warmup, k_tracked=k_tracked)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    c.close()
    f = binding.CTM(A, w.chi, precision="split_tf32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f.ctm_step(warmup + k_tracked, want_delta=False)
    E_f = f.ctm_energy(h)[1]
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    f.close()
    t_adj = max(t_grad - t_fwd, 1e-9)
    adj_flops = 3.0 * k_tracked * step_gemm_flops(w.chi, w.D2)
    return {"workload": w.name, "precision": "split_tf32 forward, FP64 QR and adjoint", "warmup": warmup,
            "k_tracked": k_tracked, "seconds": t_grad, "forward_seconds": t_fwd, "adjoint_seconds": t_adj,
            "E_site": E, "E_site_forward_only": E_f, "grad_norm": float(dA.norm().item()),
            "adjoint_fp64_tflops": adj_flops / t_adj / 1e12,
            "adjoint_frac_of_fp64_peak": adj_flops / t_adj / 1e12 / fp64_peak,
            "note": "adjoint time = ctm_grad wall time minus the forward's; frac over the whole adjoint phase"}


def optimize_record(iters=8, D=3, chi=27):
    """The variational loop (Sec. II.D): L-BFGS over the site tensor with the adjoint gradient
    (split-BF16 forward, 10 warm-up + 10 tracked steps per evaluation, each evaluation
    warm-started from the previous environment), for the Heisenberg model with the pi
    rotation on sublattice B from a seeded random D = 3 tensor at chi = 27: the energy per
    outer iteration (a variational upper bound of the QMC -0.544553) and the wall time."""
    import torch
    from paper_2509_05090_gb300 import autograd, inputs, optimize
    h = inputs.bond_hamiltonians(0.0, 1.0, rotate_b=True)
    A0 = inputs.random_site_tensor(2, D, 2024)
    autograd.release_contexts()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, energies = optimize.optimize(A0, chi, h, steps=iters, warmup=10, k_tracked=10, precision="split_bf16")
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    autograd.release_contexts()
    return {"model": "Heisenberg, B sublattice rotated", "d": 2, "D": D, "chi": chi, "seed": 2024,
            "outer_iterations": iters, "energies": energies, "seconds": secs, "seconds_per_iteration": secs / iters}


def complex_record(steps, n_split, fp64_peak, bf16_peak, with_oracle=True):
    """The complex (E-irrep) path, Kitaev K = -1 at D = 6, chi = 72 (complex enlarged corner
    2592 x 2592, the size of the real benchmark workload): steps/s in split BF16 and FP64 on the random tensor (CUDA events over one
    replayed one-step graph per step, after warm-up), then the converging tensor's time to
    delta < 1e-10 and its energy against the complex oracle."""
    import numpy as np
    import torch
    from paper_2509_05090_gb300 import binding, inputs
    w = inputs.WORKLOADS["kitaev_E_D6_chi72"]
    flops = 4.0 * step_gemm_flops(w.chi, w.D2)     # a complex product is four real ones
    rec = {"workload": w.name, "d": w.d, "D": w.D, "chi": w.chi, "n": w.n, "algorithmic_flops_per_step": flops}
    for prec in ("split_bf16", "fp64"):
        g = binding.CTMComplex(w.site_tensor(), w.chi, precision=prec, n_split=n_split)
        for _ in range(3):
            g.ctm_complex_step(1, want_delta=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = binding.ctm_kernel_launches()
        e0.record(g.stream)
        g.ctm_complex_step(steps, want_delta=False)
        e1.record(g.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        launches = (binding.ctm_kernel_launches() - l0) / steps
        g.close()
        r = {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "kernels_per_step": launches,
             "fp64_equivalent_tflops_step": flops / (ms / 1e3) / 1e12}
        if prec == "fp64":
            r["step_frac_of_fp64_peak"] = r["fp64_equivalent_tflops_step"] / fp64_peak
        else:
            pairs = n_split * (n_split + 1) // 2
            r["tensor_tflops_step"] = pairs * flops / (ms / 1e3) / 1e12
            r["step_frac_of_bf16_burst"] = r["tensor_tflops_step"] / bf16_peak
        rec[prec] = r
    wc = inputs.WORKLOADS["kitaev_E_D6_chi72_conv"]
    h = inputs.bond_hamiltonians(wc.K, wc.J, wc.d).astype(np.complex128)
    conv = {}
    for prec in ("split_bf16", "fp64"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = binding.CTMComplex(wc.site_tensor(), wc.chi, precision=prec, n_split=n_split)
        nst, dl, ok = g.ctm_complex_converge(wc.steps, wc.tol, 1)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        eb, E, _ = g.ctm_complex_energy(h)
        conv[prec] = {"steps": nst, "delta": dl, "converged": ok, "seconds": secs, "E_site": E,
                      "e_bond": [float(x) for x in eb]}
        if prec == "split_bf16":
            # the transfer-matrix spectrum of the converged complex environment (Sec. II.C)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            lam, xi, gap, iters, sok = g.ctm_complex_transfer_spectrum(nev=3, max_iter=200, tol=1e-9)
            conv[prec]["transfer_spectrum"] = {"tol": 1e-9, "lambda": [float(x) for x in lam], "xi_bravais": xi,
                                               "ln_lambda1_over_lambda2": gap, "iterations": iters,
                                               "converged": sok, "seconds": time.perf_counter() - t1}
        g.close()
    if with_oracle:
        from oracle import complex_oracle as zorc
        t0 = time.perf_counter()
        ref = zorc.ComplexCTM(wc.site_tensor(), wc.chi)
        nst, _ = ref.converge(wc.steps, wc.tol)
        _, Ez = ref.energy(list(h))
        conv["oracle"] = {"steps": nst, "E_site": Ez, "seconds": time.perf_counter() - t0,
                          "what": "numpy complex128 oracle (oracle/complex_oracle.py), all host cores via BLAS"}
        for prec in ("split_bf16", "fp64"):
            conv[prec]["abs_err_vs_oracle"] = abs(conv[prec]["E_site"] - Ez)
    rec["converge_" + wc.name] = conv
    return rec


def run_complex(args, w):
    """A complex (E-irrep) workload as the benchmark's own line: K steps of the complex path
    (one replayed one-step graph each) timed with CUDA events after warm-up, 1 GPU."""
    import numpy as np
    import torch
    from paper_2509_05090_gb300 import binding
    torch.cuda.set_device(0)
    A = w.site_tensor()
    g = binding.CTMComplex(A, w.chi, precision=args.precision, n_split=args.n_split)
    for _ in range(args.warmup):
        g.ctm_complex_step(1, want_delta=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = binding.ctm_kernel_launches()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(g.stream)
        g.ctm_complex_step(args.steps, want_delta=False)
        e1.record(g.stream)
        torch.cuda.synchronize()
    launches = binding.ctm_kernel_launches() - l0
    ms = e0.elapsed_time(e1) / args.steps
    g.close()
    peaks, src = _peaks()
    flops = 4.0 * step_gemm_flops(w.chi, w.D2)
    if args.precision == "fp64":
        fp64_peak = binding.ctm_probe_fp64_peak()
        ach = flops / (ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                    "traffic": None, "peak_source": "measured live: DFMA throughput probe",
                    "scope": "whole step (contractions, embedded QR, corner spectrum) against the FP64 pipe"}
    else:
        pairs = args.n_split * (args.n_split + 1) // 2
        ach = pairs * flops / (ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": ach / peaks["bf16_tflops"], "traffic": None, "peak_source": f"{src} bf16 burst",
                    "scope": "whole step time (a lower bound on the contraction kernels' rate)"}
    line = {"metric": METRIC, "value": 1e3 / ms, "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128" if args.precision == "fp64" else f"bf16x{args.n_split}-split+c128",
            "data": "synthetic (seeded complex site tensor, E-irrep projected)",
            "config": {"workload": w.name, "d": w.d, "D": w.D, "chi": w.chi, "n": w.n, "irrep": "E",
                       "precision": args.precision, "parallelism": "single",
                       "l2": "timed steps back to back; per-step working set > L2"},
            "roofline": roofline, "algorithmic_flops_per_step": flops, "clocks": clk.summary(),
            "gpu_launches": int(launches)}
    if not args.no_e2e:
        A_host = torch.from_numpy(np.ascontiguousarray(A)).pin_memory()
        h_host = torch.from_numpy(np.ascontiguousarray(w.hamiltonians().astype(np.complex128))).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gz = binding.CTMComplex(A_host.to("cuda", non_blocking=True), w.chi, precision=args.precision,
                                n_split=args.n_split)
        # every step's delta read back (check_every 1; a tol no delta reaches)
        nst, _, _ = gz.ctm_complex_converge(args.steps, 1e-300, 1)
        _, es, rho = gz.ctm_complex_energy(h_host.to("cuda", non_blocking=True))
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        gz.close()
        assert nst == args.steps
        t1 = time.perf_counter()
        gs = binding.CTMComplex(A_host.to("cuda", non_blocking=True), w.chi, precision=args.precision,
                                n_split=args.n_split)
        for _ in range(args.steps):
            gs.ctm_complex_step(1, want_delta=True)
        gs.ctm_complex_energy(h_host.to("cuda", non_blocking=True))
        torch.cuda.synchronize()
        t_calls = time.perf_counter() - t1
        gs.close()
        line["e2e"] = {"value": args.steps / t, "unit": "steps/s",
                       "h2d_bytes_per_step": (A_host.numel() + h_host.numel()) * 16 / args.steps,
                       "d2h_bytes_per_step": 8 + (4 + 2 * rho.size) * 8 / args.steps, "E_site": es,
                       "what": "H2D of the tensor and bond operators, init, ctm_complex_converge over K steps "
                               "with every step's delta read back, energy read back",
                       "single_step_calls": {"value": args.steps / t_calls, "unit": "steps/s"}}
    if not args.no_cpu_baseline:
        from oracle import complex_oracle as zorc
        ref = zorc.ComplexCTM(A, w.chi)
        t0 = time.perf_counter()
        nst = 0
        while nst < 4 and time.perf_counter() - t0 < 10.0:
            ref.step()
            nst += 1
        secs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nst / secs, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{nst} numpy complex128 oracle steps of {w.name} ({secs:.1f} s, BLAS "
                                          "threads on all host cores)"}
    print(json.dumps(line), flush=True)
    return 0


def chi_sweep_record(n_split, steps=3, chis=(120, 240, 360, 480), bf16_peak=None):
    """Heisenberg D = 5 at chi = 120 ... 480 in split BF16 (the sweep of the paper's
    per-iteration runtime figure): ms per step from a replayed graph of `steps` steps, the
    profiled phases (QR on the main stream, corner spectrum on the side stream) and the
    FP64-equivalent rate of the step.  chi > 224 runs the spectrum from global memory and,
    where one SM's share of the rows does not fit shared memory, the QR from the slab."""
    import torch
    from paper_2509_05090_gb300 import binding, inputs
    out = []
    for chi in chis:
        w = inputs.WORKLOADS[f"heis_D5_chi{chi}"]
        c = binding.CTM(w.site_tensor(), w.chi, precision="split_bf16", n_split=n_split)
        c.ctm_step(1, want_delta=False)       # eager first step (autotuning)
        c.ctm_step(steps, want_delta=False)   # capture + run the graph
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(c.stream)
        c.ctm_step(steps, want_delta=False)
        e1.record(c.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ph = c.ctm_step_profiled()
        c.close()
        flops = step_gemm_flops(w.chi, w.D2)
        rec = {"workload": w.name, "chi": chi, "n": w.n, "ms_per_step": ms, "steps_per_s": 1e3 / ms,
               "fp64_equivalent_tflops": flops / (ms / 1e3) / 1e12,
               "qr_ms": ph["qr"], "spectrum_ms": ph["spectrum"], "contractions_ms": ph["gemm_kernels"]}
        # the contraction kernels' BF16 slice products (T (T + 1) / 2 per algorithmic product)
        slice_tflops = n_split * (n_split + 1) / 2 * flops / (ph["gemm_kernels"] / 1e3) / 1e12
        rec["contraction_slice_tflops"] = slice_tflops
        if bf16_peak:
            rec["contraction_frac_of_bf16_burst"] = slice_tflops / bf16_peak
        out.append(rec)
    return out


def split_step_rate(w, steps, n_split, corner="qmq", precision="split_bf16"):
    import torch
    from paper_2509_05090_gb300 import binding
    c = binding.CTM(w.site_tensor(), w.chi, precision=precision, n_split=n_split, corner=corner)
    c.ctm_step(1, want_delta=False)
    c.ctm_step(steps, want_delta=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(c.stream)
    c.ctm_step(steps, want_delta=False)
    e1.record(c.stream)
    torch.cuda.synchronize()
    c.close()
    return steps / (e0.elapsed_time(e1) / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kh_D6_chi72")
    ap.add_argument("--precision", default="split_bf16", choices=["fp64", "split_bf16", "split_tf32", "fp32_tf32"])
    ap.add_argument("--n-split", type=int, default=5)
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64/oracle/convergence sub-records")
    ap.add_argument("--no-extras", action="store_true", help="skip the D=8 and batch96 sub-records")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    from paper_2509_05090_gb300 import inputs
    if args.workload == "batch96":
        return run_batch(args)
    w = inputs.WORKLOADS[args.workload]
    if w.irrep == "E" and args.impl != "reference":
        return run_complex(args, w)
    if args.impl == "reference":
        return run_reference(args, w)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2509_05090_gb300 import binding

    ws, rank, local = dist_setup()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()

    A = w.site_tensor()
    h = w.hamiltonians()
    ctm = binding.CTM(A, w.chi, precision=args.precision, n_split=args.n_split)
    for _ in range(args.warmup):
        ctm.ctm_step(1, want_delta=False)
    # a K-step call replays one captured CUDA graph of K steps; capture it (and run
    # it once) outside the timed region
    ctm.ctm_step(args.steps, want_delta=False)
    torch.cuda.synchronize()

    # ---- timed region: K back-to-back steps (the corner spectrum of step t overlaps
    # step t+1 as in real use).  The working set of one step (three n x n FP64
    # intermediates plus packed operands, >= 0.2 GB at D=6, chi=72) exceeds the
    # 129 MB L2, so no flush is inserted between steps.
    stream = ctm.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = binding.ctm_kernel_launches()
    wall0 = time.perf_counter()
    with ClockSampler(dev_index) as clk:
        e0.record(stream)
        ctm.ctm_step(args.steps, want_delta=False)
        e1.record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = binding.ctm_kernel_launches() - launches0
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, = max_over_ranks([e0.elapsed_time(e1)], ws)
    value, ms_per_step = replica_throughput(total_ms, args.steps, ws)

    # ---- profiled steps (same kernels, events between phases and around every
    # contraction launch; L2 flushed before each) for the roofline of the
    # dominant kernel, the contraction engine
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    phases = {p: 0.0 for p in binding.CTM.PHASES + binding.CTM.SIDE_PHASES}
    nprof = max(3, min(args.steps, 10))
    for _ in range(nprof):
        flush.fill_(1)
        ph = ctm.ctm_step_profiled()
        for k, v in ph.items():
            phases[k] += v
    peaks, src = _peaks()
    fp64_peak = binding.ctm_probe_fp64_peak()
    kern_ms = phases["gemm_kernels"] / nprof
    prepass_ms = phases["prepass"] / nprof
    flops = step_gemm_flops(w.chi, w.D2)
    if args.precision == "fp64":
        achieved = flops / (kern_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": None,
                    "kernel": "gemm_f64_kernel (+ split-K reduce): the step's 11 FP64 contractions",
                    "peak_source": "measured live: DFMA throughput probe (ctm_probe_fp64_peak); GB300 has no "
                                   "FP64 tcgen05 kind, so the DFMA pipe is the FP64 ceiling"}
    elif args.precision in ("split_tf32", "fp32_tf32"):
        # TF32 products on the tensor pipe: 3 (A_hi B_hi + A_hi B_lo + A_lo B_hi) or 1 per
        # contraction; the TF32 peak is the measured BF16 burst times the nominal dense ratio
        # 1.1 / 2.25 PFLOP/s
        prods = 3 if args.precision == "split_tf32" else 1
        peak = peaks["bf16_tflops"] * 1.1 / 2.25
        achieved = prods * flops / (kern_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None,
                    "kernel": f"gemm_tf32_kernel: {prods} TF32 products per contraction, tcgen05 kind::tf32 into TMEM",
                    "peak_source": f"{src} bf16 burst x 1.1/2.25 (nominal TF32/BF16 dense ratio)",
                    "fp64_equivalent_tflops": flops / (kern_ms / 1e3) / 1e12,
                    "with_prepass": {"ms_per_step": kern_ms + prepass_ms,
                                     "achieved": prods * flops / ((kern_ms + prepass_ms) / 1e3) / 1e12,
                                     "frac": prods * flops / ((kern_ms + prepass_ms) / 1e3) / 1e12 / peak}}
    else:
        T = args.n_split
        pairs = T * (T + 1) // 2
        achieved = pairs * flops / (kern_ms / 1e3) / 1e12
        peak = peaks["bf16_tflops"]
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None,
                    "kernel": f"gemm_split_kernel: {pairs} BF16 slice products (T={T}) per contraction, tcgen05 "
                              "kind::f16 into TMEM",
                    "peak_source": f"{src} bf16 burst",
                    "fp64_equivalent_tflops": flops / (kern_ms / 1e3) / 1e12,
                    "with_prepass": {"ms_per_step": kern_ms + prepass_ms,
                                     "achieved": pairs * flops / ((kern_ms + prepass_ms) / 1e3) / 1e12,
                                     "frac": pairs * flops / ((kern_ms + prepass_ms) / 1e3) / 1e12 / peak}}
    key = (w.name, args.precision, args.n_split if args.precision != "fp64" else 0)
    if key in NCU_TRAFFIC:
        roofline["traffic"] = NCU_TRAFFIC[key]
        roofline["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum of the step's 11 contraction "
                                    "launches (bytes per step, like achieved), one ncu capture, cold cache")
    roofline["kernel_ms_per_step"] = kern_ms
    roofline["prepass_ms_per_step"] = prepass_ms
    roofline["algorithmic_flops_per_step"] = flops
    roofline["phase_ms"] = {k: v / nprof for k, v in phases.items()}

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "split_tf32": "tf32x3-split+f64", "fp32_tf32": "tf32+f64"}.get(
            args.precision, f"bf16x{args.n_split}-split+f64"),
        "data": "synthetic (seeded uniform[-1,1] site tensor, C3v-projected)",
        "config": {"workload": w.name, "d": w.d, "D": w.D, "chi": w.chi, "n": w.n,
                   "precision": args.precision, "n_split": args.n_split if args.precision != "fp64" else None,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "timed steps back to back; per-step working set > L2 (no flush); profiled steps flush "
                         "256 MB before each"},
        "roofline": roofline,
        "fp64_peak_measured_tflops": fp64_peak,
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "wall_s_timed_region": wall,
    }
    ctm.close()

    # ---- mixed vs FP64 on the same GPU, and both against the FP64 oracle
    if not args.no_compare and rank == 0:
        line["mixed_vs_fp64"] = {"fp64_steps_per_s": fp64_step_record(w, args.steps, fp64_peak)["steps_per_s"]}
        e_steps = 3
        E_mix, E_orc = energy_vs_oracle(w, args.precision, args.n_split, e_steps)
        E_64, _ = energy_vs_oracle(w, "fp64", args.n_split, e_steps) if args.precision != "fp64" else (E_mix, E_orc)
        line["mixed_vs_fp64"].update({
            "after_steps": e_steps, "E_site_oracle": E_orc, "E_site_mixed": E_mix, "E_site_fp64": E_64,
            "abs_energy_error_mixed_vs_oracle": abs(E_mix - E_orc), "abs_energy_error_fp64_vs_oracle": abs(E_64 - E_orc),
            "abs_energy_error_mixed_vs_fp64": abs(E_mix - E_64)})
        # time to a converged environment on the converging stand-in at the same size
        wc = inputs.WORKLOADS.get(w.name + "_conv")
        if wc is not None:
            from oracle import oracle as orc
            conv = {"workload": wc.name, "tol": wc.tol,
                    "mixed": time_to_converged(wc, args.precision, args.n_split, wc.steps, spectrum=True),
                    "fp64": time_to_converged(wc, "fp64", args.n_split, wc.steps)}
            orc.set_threads(os.cpu_count() or 1)
            ref = orc.OracleCTM(wc.site_tensor(), wc.chi)
            t0 = time.perf_counter()
            rsteps, rdelta = ref.converge(wc.steps, wc.tol)
            rsecs = time.perf_counter() - t0
            E_ref = ref.energy(wc.hamiltonians())[1]
            conv["oracle"] = {"steps": rsteps, "delta": rdelta, "seconds": rsecs, "E_site": E_ref,
                              "threads": os.cpu_count()}
            for k in ("mixed", "fp64"):
                conv[k]["abs_energy_error_vs_oracle"] = abs(conv[k]["E_site"] - E_ref)
            line["time_to_converged"] = conv
            # the cheap corner variant C' = sym(R S) (corner_mode 1): step rate, and the
            # converged energy on the converging state against the standard oracle
            cr = time_to_converged(wc, args.precision, args.n_split, wc.steps, corner="r")
            cr["abs_energy_error_vs_oracle"] = abs(cr["E_site"] - E_ref)
            line["corner_from_r"] = {"steps_per_s": split_step_rate(w, args.steps, args.n_split, corner="r")
                                     if args.precision != "fp64" else None,
                                     "time_to_converged": cr}

    # ---- the spec D = 8, chi = 128 step in FP64 (and split for context), and the batch
    if not args.no_extras and rank == 0 and w.name == "kh_D6_chi72":
        w8 = inputs.WORKLOADS["kh_D8_chi128"]
        rec8 = fp64_step_record(w8, 3, fp64_peak)
        rec8["split_bf16_steps_per_s"] = split_step_rate(w8, 3, args.n_split)
        line["fp64_d8_chi128"] = rec8
        # the TF32 tensor-core modes: steps/s and the energy after 3 steps against the oracle
        tf = {}
        for prec in ("split_tf32", "fp32_tf32"):
            E_t, E_o = energy_vs_oracle(w, prec, args.n_split, 3)
            tf[prec] = {"steps_per_s": split_step_rate(w, args.steps, args.n_split, precision=prec),
                        "E_site_after_3_steps": E_t, "abs_err_vs_oracle": abs(E_t - E_o)}
        line["tf32_modes"] = tf
        line["grad_d8_chi128"] = grad_record(fp64_peak)
        line["optimize_heisenberg_D3"] = optimize_record()
        line["chi_sweep_heisenberg_D5"] = chi_sweep_record(args.n_split, bf16_peak=peaks["bf16_tflops"])
        line["batch96"] = batch_record(args, args.steps)
        line["complex_E_D6_chi72"] = complex_record(args.steps, args.n_split, fp64_peak, peaks["bf16_tflops"],
                                                    with_oracle=not args.no_compare)

    # end to end through the public API from pinned host memory
    if not args.no_e2e:
        A_host = torch.from_numpy(np.ascontiguousarray(w.site_tensor())).pin_memory()
        h_host = torch.from_numpy(np.ascontiguousarray(h)).pin_memory()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        A_dev = A_host.to("cuda", non_blocking=True)
        h_dev = h_host.to("cuda", non_blocking=True)
        e2e = binding.CTM(A_dev, w.chi, precision=args.precision, n_split=args.n_split)
        # ctm_converge with every step's delta read back (check_every = 1; a tol no
        # delta reaches, so exactly K steps)
        nst, _, _ = e2e.ctm_converge(max_steps=args.steps, tol=1e-300, check_every=1)
        eb, es, rho = e2e.ctm_energy(h_dev)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e.close()
        assert nst == args.steps
        # the same through K single-step calls (each returns its delta)
        t1 = time.perf_counter()
        A_dev = A_host.to("cuda", non_blocking=True)
        h_dev = h_host.to("cuda", non_blocking=True)
        e2s = binding.CTM(A_dev, w.chi, precision=args.precision, n_split=args.n_split)
        for _ in range(args.steps):
            e2s.ctm_step(1, want_delta=True)
        e2s.ctm_energy(h_dev)
        torch.cuda.synchronize()
        t_calls = time.perf_counter() - t1
        e2s.close()
        t_e2e, t_calls = max_over_ranks([t_e2e, t_calls], ws)
        line["e2e"] = {"value": ws * args.steps / t_e2e, "unit": "steps/s",
                       "h2d_bytes_per_step": (A_host.numel() * 8 + h_host.numel() * 8) / args.steps,
                       "d2h_bytes_per_step": 8 + (4 + rho.size) * 8 / args.steps,
                       "what": "H2D of the site tensor and bond operators, ctm_init, ctm_converge over K steps "
                               "with every step's delta read back (check_every 1), ctm_energy read back",
                       "E_site": es,
                       "single_step_calls": {"value": ws * args.steps / t_calls, "unit": "steps/s",
                                             "what": "the same with K ctm_step(1) calls, each returning its delta"}}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, nsteps, secs, _, _ = cpu_oracle_rate(w, budget_s=10.0, max_steps=4, threads=1)
        rate_all, nsteps_all, secs_all, _, used = cpu_oracle_rate(w, budget_s=10.0, max_steps=8, threads=0)
        line["cpu_baseline"] = {"value": rate_all, "unit": "steps/s", "cores": used, "host_cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"{nsteps_all} plain-C FP64 oracle steps of {w.name} from the initial "
                                          f"environment ({secs_all:.1f} s, {used} OpenMP threads)",
                                "single_thread": {"value": rate, "unit": "steps/s", "cores": 1,
                                                  "sample": f"{nsteps} steps ({secs:.1f} s)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
