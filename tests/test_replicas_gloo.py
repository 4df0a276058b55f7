"""The multi-process host logic (replica timing, whole-job throughput, instance
sharding) with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

from paper_2005_05436_gb300 import inputs as I  # noqa: E402
from paper_2005_05436_gb300 import replicas as R  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = R.env()
        assert (r, lr, w) == (rank, rank, world)
        # each rank "measured" a different time; the job is as slow as the slowest
        t_max = R.max_over_ranks(1.0 + rank, world)
        steps = R.sum_over_ranks(5, world)
        rate = R.whole_job_rate(steps, t_max)
        # the batch shares: every instance once, balanced by elements
        insts = I.batched_instances(64, seed=3, nelx_range=(20, 120))
        costs = [q.nelx * q.nely for q in insts]
        parts = R.shard(costs, world)
        mine = parts[rank]
        tot = R.sum_over_ranks(sum(costs[i] for i in mine), world)
        n = R.sum_over_ranks(len(mine), world)
        q.put((rank, t_max, steps, rate, tot, n, [sum(costs[i] for i in p) for p in parts], sum(costs)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, steps, rate, tot, n, loads, total in out:
        assert t_max == 2.0 and steps == 10 and rate == pytest.approx(5.0)
        assert tot == total and n == 64
        assert max(loads) - min(loads) <= max(loads) * 0.05  # within 5 %


def test_shard_single_rank_and_edge_cases():
    assert R.shard([3, 1, 2], 1) == [[0, 1, 2]]
    parts = R.shard([5, 5, 5, 5, 1], 2)
    assert sorted(parts[0] + parts[1]) == [0, 1, 2, 3, 4]
    assert R.shard([], 3) == [[], [], []]
    assert R.max_over_ranks(3.5, 1) == 3.5 and R.whole_job_rate(10, 0) == 0.0
