"""bench.py's multi-rank aggregation on CPU: two gloo ranks, each with its
own timing, agree on the slowest rank's time and the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        seconds = [2.0, 5.0][rank]            # rank 1 is the slow one
        t = bench.max_over_ranks(seconds, world)
        rate = bench.whole_job_rate(10, world, t)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [5.0, 5.0]
    assert [r[2] for r in res] == [4.0, 4.0]   # 10 units on each of 2 ranks in 5 s


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(6, 1, 3.0) == 2.0


def test_lpt_split_of_a_batch_covers_every_pair_once_and_balances():
    import bench
    rng = __import__("numpy").random.default_rng(0)
    costs = list(rng.lognormal(mean=10.0, sigma=1.0, size=256))
    for world in (2, 3, 4, 8):
        parts = bench.lpt_partition(costs, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[k] for k in p) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest pair
        assert max(loads) <= sum(costs) / world + max(costs)
        assert bench.lpt_partition(costs, world) == parts      # deterministic
    assert bench.lpt_partition([5.0, 3.0, 3.0, 2.0, 2.0], 2) == [[0, 3], [1, 2, 4]]


def _split_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        costs = [float((7 * k) % 23 + 1) for k in range(40)]
        mine = bench.lpt_partition(costs, world)[rank]
        # every rank computes the same split: gather the shares and compare
        shares = [None] * world
        dist.all_gather_object(shares, mine)
        out.put((rank, shares))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_a_batch_without_overlap():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == res[1][1]
    a, b = res[0][1]
    assert not set(a) & set(b) and sorted(a + b) == list(range(40))
