"""The multi-GPU path is N independent replicas: the method has no exchange step
(instances are independent), so `bench.py --gpus N` runs one instance per GPU with no
collective on the data path, and only the timing meets across ranks.  Its host-side
pieces are tested here on the CPU with two gloo ranks: the maximum of each timing over
the ranks (the job is as slow as its slowest replica), the whole-job throughput built
from it, and the reference arm's rank-0-only run."""
import argparse
import contextlib
import io
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench.max_over_ranks([10.0 + 5.0 * rank, 3.0 - rank], ws, device="cpu")
        value, ms = bench.replica_throughput(got[0], 20, ws)
        q.put((rank, got, value, ms))
    finally:
        dist.destroy_process_group()


def test_timings_meet_at_their_maximum_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value, ms in results:
        assert got == [15.0, 3.0]                # rank 1's 15 ms and rank 0's 3 ms
        assert abs(value - 2 * 20 / 15e-3) < 1e-9   # both replicas' steps over the slowest time
        assert abs(ms - 0.75) < 1e-12


def test_one_rank_is_the_identity():
    assert bench.max_over_ranks([4.0, 2.5], 1) == [4.0, 2.5]
    value, ms = bench.replica_throughput(8.0, 16, 1)
    assert abs(value - 2000.0) < 1e-9 and abs(ms - 0.5) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank other than 0 exits at once, printing nothing (the oracle
    is timed on the host cores once, by rank 0)."""
    from paper_2509_05090_gb300 import inputs
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=3, warmup=3)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        rc = bench.run_reference(args, inputs.WORKLOADS["kh_D6_chi72"])
    assert rc == 0 and out.getvalue() == ""


def test_reference_arm_line_times_k_steps_after_w(monkeypatch):
    """Alone (rank 0 of 1) the reference arm prints one JSON line: the oracle timed over
    exactly K steps after W untimed ones, with the keys the contract asks of that arm."""
    import json
    from paper_2509_05090_gb300 import inputs
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    args = argparse.Namespace(gpus=1, steps=2, warmup=3)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        rc = bench.run_reference(args, inputs.WORKLOADS["heis_D2_chi8"])
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    assert rc == 0 and line["impl"] == "reference"
    assert line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
