"""The multi-rank host path on CPU: two gloo ranks shard independent SpMVs
without communicating, agree on the partition, and reduce step times to the
slowest rank, as bench.py does under torchrun."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2603_04742_gb300 import dist as D  # noqa: E402


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = D.shard(costs, rank, world)
    # each rank's own "step time"; the job's time is the slowest rank's
    ms = 10.0 + 5.0 * rank
    ms_max = D.max_over_ranks(ms)
    # every rank reports its shard; gather to check disjoint cover
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    q.put((rank, mine, ms_max, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    costs = [7, 3, 9, 1, 4, 4, 8, 2, 6, 5]
    world = 2
    port = 29500 + (os.getpid() % 1000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    shards = [o[1] for o in out]
    assert sorted(shards[0] + shards[1]) == list(range(len(costs)))
    assert not set(shards[0]) & set(shards[1])
    assert all(o[3] == shards for o in out)             # everyone agrees
    assert all(o[2] == 15.0 for o in out)               # max over ranks
    loads = [sum(costs[i] for i in s) for s in shards]
    assert abs(loads[0] - loads[1]) <= max(costs)       # balanced
    assert D.aggregate_throughput([len(s) for s in shards], 15.0) == pytest.approx(
        len(costs) * 1000.0 / 15.0)


def test_shard_single_rank_is_everything():
    assert D.shard([3, 1, 2], 0, 1) == [0, 1, 2]
    assert D.max_over_ranks(2.5) == 2.5
