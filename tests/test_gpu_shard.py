"""Point-sharded seeding on the GPU (kpp_shard_* through the C ABI): several
shards of one problem -- contiguous row ranges, as Algorithm 2 partitions the
points -- each with its own kernels, workspace and buffers, all on this GPU,
with the two exchanges per pass done between them in this process
(multi.InProcessComm; between GPUs they are NCCL collectives).  The result
must be the FP64 oracle's: bit-identical on integer coordinates, within the
FP32 tolerances and the draw band otherwise, and equal to the single-call
streamed seeding's wherever the two make the same draws."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen, multi

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _store(x_np, dtype):
    x = torch.from_numpy(x_np).to(DEV)
    if dtype == "f32":
        return x, None, x_np, None
    if dtype == "bf16":
        q = kpp.quantize(x, "bf16")
        return q, None, q.cpu().numpy().view(np.uint16), None
    q, s = kpp.quantize(x, "fp8")
    return q, s, q.cpu().numpy(), s.cpu().numpy()


def run_sharded(stored, scales, K, seed, rows, dtype="f32", stream_id=0, opts=None):
    N = stored.shape[0]
    world = len(rows)
    # each shard owns its rows in an allocation of its own (16-byte aligned),
    # as a process holding one range of a problem does
    shards = [kpp.PointShard(stored[lo:hi].clone(), lo, N, K, seed, stream_id, r, world,
                             dtype=dtype,
                             row_scales=None if scales is None else scales[lo:hi].clone(),
                             opts=opts)
              for r, (lo, hi) in enumerate(rows)]
    multi.seed_sharded(shards, multi.InProcessComm(), K)
    torch.cuda.synchronize()
    idx = [s.idx.cpu().numpy() for s in shards]
    for other in idx[1:]:
        assert np.array_equal(other, idx[0])  # every shard holds the same indices
    phis = [float(s.phi.cpu()[0]) for s in shards]
    assert all(p == phis[0] for p in phis)
    d2 = np.concatenate([s.d2.cpu().numpy() for s in shards])
    return idx[0], d2, phis[0], [s.status() for s in shards]


@pytest.mark.parametrize("world", [1, 2, 3, 5])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("N,d,K", [(20_011, 16, 40), (60_000, 128, 24), (9_999, 5, 30),
                                   (4_097, 2, 64)])
def test_sharded_integer_regime_bit_identical(N, d, K, dtype, world):
    x = datagen.integer_points(N, d, seed=N + d, n_comp=8)
    stored, scales, st_np, _ = _store(x, dtype)
    idx, d2, phi, status = run_sharded(stored, scales, K, 17, multi.shard_rows(N, world), dtype)
    assert all(s == kpp.OK for s in status)
    parity.check(st_np, K, 17, 0, idx, d2, phi, exact=True)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("world", [2, 4])
def test_sharded_float_regime(world, dtype):
    x = datagen.gmm(150_001, 32, 48, seed=3)
    stored, scales, st_np, sc_np = _store(x, dtype)
    idx, d2, phi, status = run_sharded(stored, scales, 48, 2, multi.shard_rows(len(x), world),
                                       dtype)
    assert all(s == kpp.OK for s in status)
    assert parity.check(st_np, 48, 2, 0, idx, d2, phi, scales=sc_np) <= 1
    # the single-call streamed seeding: same D^2 wherever it made the same draws
    sidx, sd2, sphi = kpp.seed(stored, 48, 2, dtype=dtype, row_scales=scales,
                               opts={"form": kpp.FORM_STREAMED})
    if np.array_equal(sidx.cpu().numpy(), idx):
        assert np.array_equal(sd2.cpu().numpy(), d2)


def test_uneven_shards_and_a_one_row_shard():
    N = 30_000
    x = datagen.integer_points(N, 8, seed=4, n_comp=6)
    rows = [(0, 1), (1, 7_000), (7_000, 7_001), (7_001, 29_999), (29_999, N)]
    idx, d2, phi, status = run_sharded(torch.from_numpy(x).to(DEV), None, 50, 3, rows)
    parity.check(x, 50, 3, 0, idx, d2, phi, exact=True)


def test_sharded_exact_draws_and_stream_id():
    x = datagen.gmm(80_000, 16, 24, seed=7)
    xs = torch.from_numpy(x).to(DEV)
    rows = multi.shard_rows(len(x), 3)
    a = run_sharded(xs, None, 24, 5, rows, stream_id=4)
    b = run_sharded(xs, None, 24, 5, rows, stream_id=4, opts={"exact_draws": 1})
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    assert parity.check(x, 24, 5, 4, a[0], a[1], a[2]) <= 1


def test_sharded_degenerate_data():
    base = np.array([[0, 0, 0, 0], [1, 2, 3, 4], [5, 5, 5, 5]], np.float32)
    x = np.repeat(base, [400, 300, 301], axis=0)
    x = x[np.random.default_rng(0).permutation(len(x))]
    idx, d2, phi, status = run_sharded(torch.from_numpy(x).to(DEV), None, 5, 1,
                                       multi.shard_rows(len(x), 3))
    assert all(s == kpp.ERR_DEGENERATE for s in status)
    assert np.all(idx[3:] == -1)
    parity.check(x, 5, 1, 0, idx, d2, phi, exact=True, status=oracle.DEGENERATE)


def test_sharded_argument_errors():
    x = torch.zeros((100, 4), device=DEV)
    with pytest.raises(kpp.KppError):
        kpp.PointShard(x, 50, 120, 4, 1, 0, 0, 2)  # rows past n_global
    with pytest.raises(kpp.KppError):
        kpp.PointShard(x, 0, 100, 4, 1, 0, 2, 2)  # rank >= world
    s = kpp.PointShard(x, 0, 100, 4, 1, 0, 0, 1)
    assert kpp.kpp_shard_pass(s.desc, 4, s.exchange.data_ptr(), s.total.data_ptr(),
                              kpp._stream_handle(torch.device(DEV))) == kpp.ERR_INVALID_ARG
    assert kpp.kpp_shard_pick(s.desc, 3, s.totals.data_ptr(), s.exchange.data_ptr(),
                              kpp._stream_handle(torch.device(DEV))) == kpp.ERR_INVALID_ARG


_NCCL_CHILD = r"""
import os, sys, numpy as np, torch, torch.distributed as dist
sys.path.insert(0, os.getcwd())
import oracle
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen, multi
dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda:0"))
x = datagen.integer_points(30_011, 16, seed=3, n_comp=8)
lo, hi = multi.shard_rows(len(x), 1)[0]
s = kpp.PointShard(torch.from_numpy(x[lo:hi]).to("cuda:0"), lo, len(x), 24, 5, 0, 0, 1)
multi.seed_sharded([s], multi.ProcessGroupComm(dist), 24)
torch.cuda.synchronize()
ref = oracle.seed(x, 24, 5, 0)
assert s.status() == kpp.OK
assert np.array_equal(s.idx.cpu().numpy(), ref["idx"])
assert np.array_equal(s.d2.cpu().numpy().astype(np.float64), ref["d2"])
assert float(s.phi.cpu()[0]) == ref["phi"]
dist.destroy_process_group()
print("nccl protocol ok")
"""


def test_protocol_over_nccl_on_one_rank():
    """The exchanges as NCCL collectives through torch.distributed (a
    one-rank group: the process-group path the multi-GPU run takes, on the
    one GPU here), bit-identical to the oracle on integer data."""
    import os
    import subprocess
    import sys

    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(29500 + os.getpid() % 1000))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _NCCL_CHILD], capture_output=True, text=True,
                       cwd=root, env=env, timeout=600)
    assert r.returncode == 0 and "nccl protocol ok" in r.stdout, r.stdout[-2000:] + r.stderr[-3000:]
