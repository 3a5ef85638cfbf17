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


# ---------------------------------------------------------------------------
# One problem sharded by points (Algorithm 2's partition N_1 .. N_l, one
# contiguous range of rows per GPU).  Per pass the shards exchange two small
# messages: an all-gather of their D^2 totals (two floats each) and a sum of
# their exchange buffers (the owner of the new centre contributes its row,
# the others zeros).  No host synchronisation happens between passes.
# ---------------------------------------------------------------------------


def shard_rows(N: int, world: int):
    """Contiguous row ranges [lo, hi) of ``world`` shards of N rows, in rank
    order (the first N % world shards one row longer)."""
    if world < 1 or N < world:
        raise ValueError("need 1 <= world <= N")
    base, extra = divmod(N, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def seed_sharded(shards, comm, K: int):
    """The seeding of one problem over point shards.

    ``shards``: the shards this process drives (one per process in a
    multi-process run; all of them when every shard lives in this process),
    each with ``first()``, ``local_pass(m)``, ``pick(m)``, ``finish()`` and the
    buffers ``exchange`` (summed), ``total`` (gathered into ``totals``).
    ``comm``: ``sum(buffers)`` and ``gather(parts, outs)`` over all shards.
    """
    for s in shards:
        s.first()
    comm.sum([s.exchange for s in shards])
    for m in range(K):
        for s in shards:
            s.local_pass(m)
        comm.gather([s.total for s in shards], [s.totals for s in shards])
        if m < K - 1:
            for s in shards:
                s.pick(m)
            comm.sum([s.exchange for s in shards])
    for s in shards:
        s.finish()


class ProcessGroupComm:
    """One shard per process: the exchanges as torch.distributed collectives
    (NCCL between GPUs, gloo between CPU processes)."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group

    def sum(self, bufs):
        (b,) = bufs
        self.dist.all_reduce(b, op=self.dist.ReduceOp.SUM, group=self.group)

    def gather(self, parts, outs):
        import torch

        (p,), (o,) = parts, outs
        world = self.dist.get_world_size(self.group)
        got = [torch.empty_like(p) for _ in range(world)]
        self.dist.all_gather(got, p, group=self.group)
        o.copy_(torch.cat(got))


class InProcessComm:
    """Every shard in this process (e.g. several shards on one GPU): the same
    exchanges as tensor copies -- the sum of the exchange buffers and the
    concatenation of the totals in rank order."""

    def sum(self, bufs):
        total = bufs[0].clone()
        for b in bufs[1:]:
            total += b
        for b in bufs:
            b.copy_(total)

    def gather(self, parts, outs):
        import torch

        g = torch.cat(list(parts))
        for o in outs:
            o.copy_(g)
