"""Host logic of the multi-GPU bench path, on CPU with the gloo backend.

The propagation shards over independent domains, so N GPUs run N replicas
with no data exchanged; the only collective is the max-over-ranks of the
timed region, and the job's throughput is N replicas' units over the slowest
rank's time.  These run as two gloo ranks on the host; no GPU is touched.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        t = bench._max_over_ranks(10.0 + 3.0 * rank, ws)    # rank r was timed at 10 + 3 r seconds
        v = bench._job_value(ws, 1000.0, t)
        dist.barrier()
        q.put((rank, t, v, bench._dist()))
    finally:
        dist.destroy_process_group()


def test_replicas_time_is_the_slowest_rank_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, d in out:
        assert t == 13.0                          # every rank reports the slowest time
        assert v == pytest.approx(2 * 1000.0 / 13.0)
        assert d == (ws, rank, rank)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(4.5, 1) == 4.5
    assert bench._job_value(1, 900.0, 3.0) == 300.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle; the others return at once
    without work and print nothing."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 1, 2

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
