"""GPU paths that the workload-driven tests reach only by chance.

* Every contraction tile width of the split engine (48: two CTAs per SM, 64, 96),
  forced through the plan cache (CTM_AUTOTUNE_CACHE) in a fresh process per width,
  for a whole CTMRG step against the FP64 oracle.
* The blocked QR's early panel end: a previous projector with nearly parallel
  column pairs makes the reduced corner's columns nearly dependent, so downdated
  panel norms collapse and the factorisation restarts panels from fresh sums.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _step_shapes(chi, D2):
    n = chi * D2
    return sorted({(n, chi, chi), (n, n, chi), (chi * chi, D2, D2 * D2), (chi * chi, D2 * D2, D2), (n, chi, n),
                   (chi, chi, n), (chi, n, n)})


_CHILD = textwrap.dedent("""
    import sys, numpy as np
    sys.path.insert(0, sys.argv[1])
    from paper_2509_05090_gb300 import binding
    env = np.load(sys.argv[2])
    g = binding.CTM(env["A"], int(env["chi"]), precision="split_bf16", n_split=5)
    g.ctm_set_env(env["C"], env["T"], env["Q"])
    g.ctm_step(1)
    np.savez(sys.argv[3], M=g.ctm_get_intermediate("M").cpu().numpy(), s=g.ctm_get_intermediate("s").cpu().numpy())
    g.close()
""")


def _plan_line(M, N, K, nt):
    return f"split {M} {N} {K} 5 : {nt} 1\n"


@pytest.mark.parametrize("wl,nt", [("kitaev_D4_chi32", 48), ("kitaev_D4_chi32", 64), ("kitaev_D4_chi32", 96),
                                   ("kh_D6_chi72", 48)])
def test_split_step_each_tile_width(ctm_lib, tmp_path, wl, nt):
    """One split step with every contraction forced onto one plan family."""
    w = I.WORKLOADS[wl]
    A = w.site_tensor()
    ref = O.OracleCTM(A, w.chi)
    for _ in range(3 if w.chi <= 32 else 1):
        ref.step()
    env = tmp_path / "env.npz"
    np.savez(env, A=A, chi=w.chi, C=ref.C, T=ref.T, Q=ref.Q)
    ref.step()
    cache = tmp_path / "plans.txt"
    cache.write_text("".join(_plan_line(M, N, K, nt) for M, N, K in _step_shapes(w.chi, w.D2)))
    out = tmp_path / "out.npz"
    script = tmp_path / "child.py"
    script.write_text(_CHILD)
    r = subprocess.run([sys.executable, str(script), ROOT, str(env), str(out)], capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, CTM_AUTOTUNE_CACHE=str(cache)))
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(out)
    # T = 5 slices: the contraction error bound (see test_gpu_split) is far below 1e-9 of max|M|
    assert _rel(got["M"], ref.last["M"]) <= 1e-9
    assert np.max(np.abs(got["s"] - ref.s)) <= 1e-7


def test_qr_panel_restart_on_nearly_parallel_columns(ctm_lib):
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["kitaev_D4_chi32"]
    A = w.site_tensor()
    ref = O.OracleCTM(A, w.chi)
    for _ in range(3):
        ref.step()
    Q = ref.Q.copy()
    for c in (1, 9, 17, 26):   # inside panels and at a panel start
        Q[:, c] = Q[:, c - 1] + 1e-3 * Q[:, c]
    ref.set_env(ref.C, ref.T, Q)
    g = binding.CTM(A, w.chi)
    g.ctm_set_env(ref.C, ref.T, Q)
    ref.step()
    g.ctm_step(1)
    last = ref.last
    Y = last["Y"]
    # the reduced corner really has nearly dependent column pairs
    cosang = abs(Y[:, 1] @ Y[:, 0]) / (np.linalg.norm(Y[:, 1]) * np.linalg.norm(Y[:, 0]))
    assert cosang > 0.99
    R_ref = last["R"]
    dR = np.abs(np.diag(R_ref))
    lead = int(np.sum(dR / dR[0] >= 1e-8))
    R = _np(g.ctm_get_intermediate("R"))
    assert np.all(np.diag(R) >= 0.0)
    assert _rel(R[:lead], R_ref[:lead]) <= 1e-10
    C, T, Qn = (_np(x) for x in g.ctm_get_env())
    assert _rel(Qn[:, :lead], last["Q"][:, :lead]) <= 1e-10
    assert np.max(np.abs(Qn.T @ Qn - np.eye(w.chi))) <= 1e-12
    assert np.max(np.abs(Qn @ R - _np(g.ctm_get_intermediate("Y")))) <= 1e-12 * np.max(np.abs(Y))
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_forced_wait_timeout_is_reported(ctm_lib, precision):
    """Failure detection without a fault: the context's forced-timeout switch makes the
    QR grid barrier wait for an arrival that never comes; the bounded wait gives up,
    the step returns CTM_ETIMEOUT, the context can be destroyed, and a fresh context
    on the same device then steps like the oracle."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["heis_D2_chi8"]
    A = w.site_tensor()
    g = binding.CTM(A, w.chi, precision=precision, n_split=5)
    g.ctm_step(2)                      # eager first step, then a captured one
    g.ctm_debug_force_timeout(True)
    with pytest.raises(binding.CtmError) as ei:
        g.ctm_step(1)
    assert ei.value.status == 6        # CTM_ETIMEOUT
    g.close()
    # the same through ctm_converge's pipelined graphs (the error flag comes back with a
    # chunk's deltas; a chunk already queued is drained before the call returns)
    g = binding.CTM(A, w.chi, precision=precision, n_split=5)
    g.ctm_step(2)
    g.ctm_debug_force_timeout(True)
    with pytest.raises(binding.CtmError) as ei:
        g.ctm_converge(max_steps=20, tol=1e-300, check_every=2)
    assert ei.value.status == 6
    g.close()
    ref = O.OracleCTM(A, w.chi)
    g2 = binding.CTM(A, w.chi, precision=precision, n_split=5)
    for _ in range(5):
        dr = ref.step()
        dg = g2.ctm_step(1)
        assert abs(dg - dr) <= 1e-8 * max(1.0, abs(dr))
    C, T, Q = (_np(x) for x in g2.ctm_get_env())
    assert _rel(C, ref.C) <= 1e-8
    g2.close()


def _pipelined_steps(deltas, k, tol, max_steps):
    """The step count of ctm_converge(max_steps, tol, check_every=k) on a context whose
    first step is eager, given the delta of every step (deltas[i]: step i + 1): chunks
    of k steps, a second one queued behind the one being read while the newest delta
    read is above 100 tol (or unknown); a chunk shows the delta of the step before it
    (slot 0, no information in the first chunk of a run) and of its own steps but the
    last; queueing stops when the newest delta read is below tol, and a run of chunks
    ends with the last step's own spectrum.  Fewer than k steps left run one at a
    time."""
    done = 1
    if deltas[0] < tol:
        return done
    while done < max_steps:
        budget = max_steps - done
        if budget < k:
            done += 1
            if deltas[done - 1] < tol:
                return done
            continue
        queue, launched, stop, reads, newest = [], 0, False, 0, float("inf")
        while True:
            while not stop and len(queue) < (2 if newest > 100 * tol else 1) and launched + k <= budget:
                queue.append(launched)
                launched += k
            if not queue:
                break
            base = done + queue.pop(0)      # steps done before this chunk
            slots = [deltas[base - 1]] + [deltas[base + i - 1] for i in range(1, k)]
            first = 1 if reads == 0 else 0
            reads += 1
            if k - 1 >= first:
                newest = slots[k - 1]
                stop = newest < tol
        done += launched
        if deltas[done - 1] < tol:
            return done
    return done


@pytest.mark.parametrize("precision,k", [("fp64", 1), ("split_bf16", 1), ("split_bf16", 3)])
def test_pipelined_converge_matches_single_steps(ctm_lib, precision, k):
    """ctm_converge keeps one chunk of check_every steps queued behind the one whose
    deltas it reads and defers each chunk's last corner spectrum to the head of the
    next.  Against a context stepped one call at a time (delta read back after each
    step): the same environment after as many steps, the reported delta equal to that
    step's delta, and the step count that the delta sequence implies."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["heis_D2_chi8"]
    A, tol = w.site_tensor(), 1e-10
    g1 = binding.CTM(A, w.chi, precision=precision, n_split=5)
    steps, delta, ok = g1.ctm_converge(max_steps=200, tol=tol, check_every=k)
    assert ok and delta < tol
    g2 = binding.CTM(A, w.chi, precision=precision, n_split=5)
    deltas = [g2.ctm_step(1) for _ in range(steps)]
    assert _pipelined_steps(deltas, k, tol, 200) == steps
    assert abs(delta - deltas[-1]) <= 1e-13 + 1e-6 * abs(deltas[-1])
    for x, y in zip(g1.ctm_get_env(), g2.ctm_get_env()):
        assert _rel(_np(x), _np(y)) <= 1e-10
    # a step limit that is not a multiple of the chunk: exactly max_steps steps
    steps2, _, ok2 = g1.ctm_converge(max_steps=7, tol=1e-300, check_every=3)
    assert steps2 == 7 and not ok2
    g2.ctm_step(7)
    for x, y in zip(g1.ctm_get_env(), g2.ctm_get_env()):
        assert _rel(_np(x), _np(y)) <= 1e-10
    g1.close()
    g2.close()


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_deterministic_mode_gives_bitwise_equal_replays(ctm_lib, precision):
    """With cfg.deterministic the QR's cross-CTA sums are per-CTA partials added in CTA
    order (no FP64 atomics): a context stepped one call at a time and another replaying a
    captured multi-step graph reach bit-identical environments, and one step from the
    oracle's environment still matches the oracle's factorisation."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["kitaev_D4_chi32"]
    A = w.site_tensor()
    g1 = binding.CTM(A, w.chi, precision=precision, n_split=5, deterministic=True)
    g2 = binding.CTM(A, w.chi, precision=precision, n_split=5, deterministic=True)
    for _ in range(12):
        g1.ctm_step(1)
    g2.ctm_step(1)
    g2.ctm_step(11)
    for x, y in zip(g1.ctm_get_env(), g2.ctm_get_env()):
        assert np.array_equal(_np(x), _np(y))
    g1.close()
    g2.close()
    ref = O.OracleCTM(A, w.chi)
    ref.step()
    ref.step()
    g = binding.CTM(A, w.chi, precision="fp64", deterministic=True)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    g.ctm_step(1)
    ref.step()
    R_ref = ref.last["R"]
    dR = np.abs(np.diag(R_ref))
    lead = int(np.sum(dR / dR[0] >= 1e-8))
    assert lead >= w.chi // 2
    R = _np(g.ctm_get_intermediate("R"))
    assert np.max(np.abs(R[:lead, :lead] - R_ref[:lead, :lead])) <= 1e-10 * dR[0]
    g.close()


def test_converge_after_set_site_uses_the_new_tensor(ctm_lib):
    """ctm_set_site drops every captured graph (they assumed the old double layer's packed
    digits): ctm_converge after swapping in a new tensor reaches the energy of a fresh
    context on that tensor."""
    from paper_2509_05090_gb300 import binding
    w = I.WORKLOADS["heis_D2_chi8"]
    h = w.hamiltonians()
    A1 = w.site_tensor()
    A2 = I.random_site_tensor(2, 2, 4242)
    g = binding.CTM(A1, w.chi, precision="split_bf16", n_split=5)
    g.ctm_converge(max_steps=200, tol=1e-11, check_every=1)
    g.ctm_set_site(A2, reset_env=True)
    _, _, ok = g.ctm_converge(max_steps=300, tol=1e-11, check_every=1)
    E = g.ctm_energy(h)[1]
    f = binding.CTM(A2, w.chi, precision="split_bf16", n_split=5)
    _, _, okf = f.ctm_converge(max_steps=300, tol=1e-11, check_every=1)
    Ef = f.ctm_energy(h)[1]
    assert ok == okf
    assert abs(E - Ef) <= 1e-9
    g.close()
    f.close()
