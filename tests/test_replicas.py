"""Host logic of the N-replica benchmark on CPU ranks (gloo, world size 2).

The decomposition does not shard: each rank runs whole problems on its own GPU
with no collective on the data path.  What crosses ranks is the timing: a
barrier around the timed region and the maximum of the per-rank times, from
which rank 0 reports the whole-job throughput.  These tests run that logic with
gloo ranks on the CPU; no GPU is involved.
"""
import os
import socket
import sys
import types

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    cpu = torch.device("cpu")
    bench.barrier_sync(ws, cpu)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    worst = bench.max_over_ranks(local_ms, ws, cpu)
    q.put((rank, worst, bench.replica_throughput(ws, 10, worst)))
    bench.barrier_sync(ws, cpu)
    dist.destroy_process_group()


def test_two_rank_max_time_and_whole_job_throughput():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, worst, value in out:
        assert worst == 150.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 10 / 0.150)  # units of all ranks over the max time


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_oracle_worker", lambda *a, **k: called.append(a))
    args = types.SimpleNamespace(steps=1, warmup=0)
    assert bench.bench_reference(args) is None
    assert not called  # the other ranks do no work
