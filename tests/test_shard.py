"""Independent problems spread over ranks (host logic, CPU): the partition by
estimated work and the final gather to rank 0, across two real gloo
processes.  Each rank evaluates its share with the oracle in place of the
library's batch, so the gathered results can be compared exactly with an
unsharded evaluation."""
import os
import socket

import numpy as np
import pytest

from paper_2505_00529_gb300 import inputs, shard


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_batched_shape_matches_the_workload():
    for i in (0, 1, 17, 255):
        p = inputs.config_problem(3, i)
        assert inputs.batched_shape(i) == (p.N, p.K, p.J)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_problem_once_and_balances(world):
    shapes = [inputs.batched_shape(i) for i in range(256)]
    parts = shard.partition(shapes, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(256))
    assert all(p == sorted(p) for p in parts)
    load = [sum(shard.estimated_flops(*shapes[i]) for i in p) for p in parts]
    # largest-first greedy: no rank exceeds the mean by more than the largest problem
    assert max(load) - np.mean(load) <= max(shard.estimated_flops(*s) for s in shapes)
    assert max(load) / np.mean(load) < 1.05
    assert shard.partition(shapes, world) == parts            # deterministic


def test_partition_more_ranks_than_problems():
    parts = shard.partition([(8, 4, 100), (16, 4, 100)], 4)
    assert parts == [[1], [0], [], []]


def _problems():
    shapes = [(4, 3, 40), (6, 5, 33), (3, 2, 20), (8, 4, 25), (5, 6, 31)]
    probs = [inputs.small_problem(N, K, J, seed=70 + i, dt=0.05) for i, (N, K, J) in enumerate(shapes)]
    thetas = [inputs.eval_theta(p.K, 80 + i, 0.5) for i, p in enumerate(probs)]
    return probs, thetas


def _oracle_eval(probs, thetas):
    from oracle import qoc_oracle as orc
    out = []
    for p, t in zip(probs, thetas):
        r = orc.evaluate(p, t, order=2)
        out.append((r["J"], r["grad"], r["hess"]))
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        probs, thetas = _problems()
        res, mine = shard.evaluate_sharded(probs, thetas, rank, world, dist, evaluate=_oracle_eval)
        q.put((rank, mine, res))
    finally:
        dist.destroy_process_group()


def test_sharded_evaluation_gathers_to_rank0():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    (r0, mine0, res0), (r1, mine1, res1) = got
    assert res1 is None and sorted(mine0 + mine1) == list(range(5)) and mine0 and mine1
    probs, thetas = _problems()
    ref = _oracle_eval(probs, thetas)
    assert len(res0) == len(ref)
    for (J, g, H), (Jr, gr, Hr) in zip(res0, ref):
        assert J == Jr
        np.testing.assert_array_equal(g, gr)
        np.testing.assert_array_equal(H, Hr)


def test_single_rank_needs_no_process_group():
    probs, thetas = _problems()
    res, mine = shard.evaluate_sharded(probs, thetas, 0, 1, None, evaluate=_oracle_eval)
    assert mine == list(range(5)) and len(res) == 5
