"""Multi-process host logic of bench.py (replicas under torchrun), as 2 gloo ranks on the CPU.

The path shards by scene or view with no exchange, so the only cross-rank steps are the barrier
around the timed region and the maximum of the ranks' times; the whole-job rate is the steps of
all replicas over the slowest rank's time.  The reference arm runs on rank 0 alone.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

STEPS = 7


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own_ms = 100.0 + 37.5 * rank  # rank 1 is the slowest
        dist.barrier()
        ms = bench.max_over_ranks(own_ms, dist, "cpu")
        q.put((rank, ms, bench.whole_job_rate(world, STEPS, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    slowest = 137.5
    for rank, ms, rate in got:
        assert ms == slowest
        assert rate == pytest.approx(2 * STEPS / (slowest / 1000.0), rel=1e-12)


def test_single_rank_passthrough():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_rate(1, 10, 500.0) == pytest.approx(20.0)


def test_reference_arm_other_ranks_exit_without_work(capsys):
    class Args:
        steps, warmup, gpus = 1, 0, 2

    bench.reference_arm(Args, rank=1, world=2)
    assert capsys.readouterr().out == ""
