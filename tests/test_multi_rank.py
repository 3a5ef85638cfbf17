"""The host logic of running on several GPUs, tested on CPU ranks: two gloo
processes (world size 2) agree on the problem split of the batching form
without communicating, the split is disjoint, complete and balanced, and the
max/sum over ranks that combine the timings are correct."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1908_02136_gb300 import datagen, multi


def test_shard_is_a_balanced_partition():
    table = datagen.batch_table()
    costs = [pr.N * pr.K * pr.d for pr in table]
    for world in (1, 2, 3, 4, 8):
        shards = multi.shard_problems(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(table)))
        loads = multi.shard_loads(costs, shards)
        # LPT: no rank exceeds the mean by more than the largest single job
        assert max(loads) - sum(loads) / world <= max(costs) + 1e-9


def test_shard_small_cases():
    assert multi.shard_problems([], 3) == [[], [], []]
    assert multi.shard_problems([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]
    assert multi.shard_problems([1, 1], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        multi.shard_problems([1], 0)
    assert multi.replica_stream(7, 0) == 7
    assert multi.replica_stream(7, 1) != multi.replica_stream(7, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        table = datagen.batch_table()
        costs = [pr.N * pr.K * pr.d for pr in table]
        mine = multi.shard_problems(costs, world)[rank]
        # every rank's own view of the split, gathered
        views = [None] * world
        dist.all_gather_object(views, mine)
        t_max = multi.max_over_ranks(10.0 + rank, dist)
        t_sum = multi.sum_over_ranks(float(len(mine)), dist)
        q.put((rank, views, t_max, t_sum))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_split_and_the_max():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    table = datagen.batch_table()
    expect = multi.shard_problems([pr.N * pr.K * pr.d for pr in table], world)
    for rank, views, t_max, t_sum in results:
        assert views == expect  # each rank computed the same split on its own
        assert t_max == 11.0
        assert t_sum == float(len(table))
    assert set(expect[0]).isdisjoint(expect[1])


def test_without_a_process_group_the_value_passes_through():
    assert multi.max_over_ranks(3.5) == 3.5
    assert multi.sum_over_ranks(2.0) == 2.0
