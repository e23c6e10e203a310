"""Host logic of the multi-rank bench on CPU: two gloo ranks (replicas, weak
scaling) agree on the max-over-ranks time, the whole-job value counts the
units of every rank, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, e = bench.aggregate_over_ranks(1.0 + rank, 4.0 - 3.0 * rank, dist)
        out.put((rank, t, e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # rank 0: t = 1, e2e = 4; rank 1: t = 2, e2e = 1 -> both see the maxima (2, 4)
    assert got == [(0, 2.0, 4.0), (1, 2.0, 4.0)]


def test_single_rank_and_whole_job_value():
    assert bench.aggregate_over_ranks(3.5, 1.25) == (3.5, 1.25)
    # 2 ranks x 100 units per step x 5 steps in 2 s
    assert bench.whole_job_value(2, 100.0, 5, 2.0) == 500.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) is None
