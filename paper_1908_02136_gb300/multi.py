"""Host-side logic of running the seeding on several GPUs, one process each.

Both ways of using more than one GPU need no collective on the data path:

* independent problems (the batching form): the problems are split between
  the ranks, each rank seeds its share with its own kpp_seed_batched launch,
  and only the timing is combined;
* one problem per rank (replicas): every rank seeds its own copy with its
  own draw stream.

What is shared between ranks is the maximum step time (the job is as slow as
its slowest rank).  These helpers work with any torch.distributed backend
(NCCL on GPUs, gloo on CPUs in the tests).
"""
from __future__ import annotations

import heapq


def shard_problems(costs, world: int):
    """Longest-processing-time split of problems over ``world`` ranks.

    ``costs``: per-problem cost (e.g. N*K*d*bytes).  Problems are taken in
    decreasing cost (ties by index) and each goes to the rank with the least
    cost so far (ties by rank).  Returns one ascending index list per rank;
    the lists are disjoint and cover every problem.  Deterministic, so every
    rank computes the same split without communicating.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in shards]


def shard_loads(costs, shards):
    """Total cost of each rank's share."""
    return [sum(float(costs[i]) for i in s) for s in shards]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of ``value`` over all ranks (``value`` itself without a
    process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """The sum of ``value`` over all ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_stream(stream_id: int, rank: int, stride: int = 1 << 20) -> int:
    """Draw stream of rank ``rank``'s replica of a problem: distinct per rank,
    equal to ``stream_id`` on rank 0."""
    return stream_id + rank * stride
