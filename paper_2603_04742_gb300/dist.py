"""Host-side multi-GPU helpers: one process per GPU.

The method shards without a data-path exchange: chunks are independent until
the masked sum of Algorithm 4, and separate SpMVs (or row partitions) are
fully independent.  Ranks therefore take disjoint sets of SpMVs; the only
collective is the timing reduction (the slowest rank defines the step time).
"""
import os


def env_rank():
    """(rank, world, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(costs, rank, world):
    """Indices of the work units rank `rank` runs: greedy longest-first
    assignment of units with estimated `costs` (e.g. key switches per SpMV)
    to the least-loaded rank; ties go to the lower rank.  Deterministic, so
    every rank computes the same partition without communicating."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def max_over_ranks(value, device=None):
    """The maximum of a float over all ranks (identity without a process
    group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank, ms_per_step_max):
    """Whole-job throughput (units/s): all ranks' units over the slowest
    rank's step time."""
    return sum(units_per_rank) * 1000.0 / ms_per_step_max
