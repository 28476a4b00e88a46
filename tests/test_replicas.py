"""Multi-rank (replica) host logic of bench.py on CPU: world size 2 over gloo.

A single problem is one dependent chain over the time steps and does not
shard; with several processes every rank evaluates its own replica and the
job is timed by its slowest rank.  These tests run the reduction the
benchmark uses across two real processes (no GPU)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")   # rank 1 is slower
        out.put((rank, ms, bench.whole_job_rate(world, ms)))
    finally:
        dist.destroy_process_group()


def test_single_rank_is_its_own_maximum():
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(1, 4.0) == 250.0


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(out.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [r for r, _, _ in res] == [0, 1]
    for _, ms, rate in res:
        assert ms == 15.0                        # both ranks see the slowest replica
        assert rate == pytest.approx(2 * 1000.0 / 15.0, rel=1e-15)
    assert all(p.exitcode == 0 for p in procs)
