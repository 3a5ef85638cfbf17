"""Point-sharded seeding of one problem (Algorithm 2's partition of the
points into N_1 .. N_l, one contiguous row range per process), host side:
the protocol of multi.seed_sharded -- first seed, then per pass a local pass,
an all-gather of the shards' D^2 totals, the draw and a sum of the exchange
buffers -- driven around a NumPy restatement of the shard's steps on integer
coordinates, must reproduce the single-process FP64 oracle bit for bit:
in one process (every shard local) and over 2 and 3 gloo processes."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1908_02136_gb300 import datagen, multi
from shard_restatement import CpuShard


def test_shard_rows_partition():
    for N, world in [(10, 1), (10, 3), (7, 7), (100_003, 8)]:
        rows = multi.shard_rows(N, world)
        assert rows[0][0] == 0 and rows[-1][1] == N
        assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
        sizes = [hi - lo for lo, hi in rows]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        multi.shard_rows(2, 3)


def _run_local(x, K, seed, stream_id, world):
    shards = [CpuShard(x[lo:hi], lo, len(x), K, seed, stream_id, r, world)
              for r, (lo, hi) in enumerate(multi.shard_rows(len(x), world))]
    multi.seed_sharded(shards, multi.InProcessComm(), K)
    return shards


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("N,d,K", [(5_003, 8, 24), (1_001, 3, 40), (20_011, 16, 12)])
def test_in_process_shards_match_the_oracle(N, d, K, world):
    x = datagen.integer_points(N, d, seed=N + world, n_comp=8)
    shards = _run_local(x, K, 5, 0, world)
    ref = oracle.seed(x, K, 5, 0)
    for s in shards:
        assert np.array_equal(s.idx, ref["idx"])
        assert s.phi == ref["phi"]
    assert np.array_equal(np.concatenate([s.d2 for s in shards]), ref["d2"])


def test_in_process_degenerate_stop():
    base = np.array([[0, 0], [1, 2], [5, 5]], np.float32)
    x = np.repeat(base, [40, 30, 31], axis=0)
    x = x[np.random.default_rng(0).permutation(len(x))]
    shards = _run_local(x, 5, 1, 0, 3)
    ref = oracle.seed(x, 5, 1, 0)
    assert ref["status"] == oracle.DEGENERATE
    for s in shards:
        assert s.status == oracle.DEGENERATE
        assert np.array_equal(s.idx, ref["idx"])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q, N, d, K, seed):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x = datagen.integer_points(N, d, seed=N, n_comp=8)
        lo, hi = multi.shard_rows(N, world)[rank]
        s = CpuShard(x[lo:hi], lo, N, K, seed, 0, rank, world)
        multi.seed_sharded([s], multi.ProcessGroupComm(dist), K)
        q.put((rank, s.idx, s.d2, s.phi, s.status))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_the_oracle(world):
    N, d, K, seed = 12_007, 16, 32, 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, N, d, K, seed))
             for r in range(world)]
    for p in procs:
        p.start()
    results = sorted([q.get(timeout=180) for _ in range(world)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = datagen.integer_points(N, d, seed=N, n_comp=8)
    ref = oracle.seed(x, K, seed, 0)
    for rank, idx, d2, phi, status in results:
        assert status == oracle.OK
        assert np.array_equal(idx, ref["idx"])
        assert phi == ref["phi"]
    assert np.array_equal(np.concatenate([r[2] for r in results]), ref["d2"])
