"""GPU parity at the full sizes of the precision workloads (10^7 x 64 with
K = 1024, and 2*10^7 x 128 with K = 2048), in the forms the autotuner picks
for them, on outputs the FP64 oracle can check one at a time:

* the first seed against floor(u_0 * N);
* D^2 of 2000 sampled rows against the FP64 minimum over all K chosen
  centres (the stored values decoded exactly), 1e-5 relative;
* sampled draws: a seeding stopped after m seeds returns the D^2 the full
  run drew seed m from (same seed, same trajectory), so the oracle's FP64
  inverse CDF on that array must give the full run's index m (or a counted
  near-boundary event);
* properties that hold at any size: distinct indices in range, D^2 = 0 at
  every chosen point, phi = sum D^2.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEV = "cuda:0"
SEED = 1


def _decode(stored, scales, dtype, rows):
    """FP64 values of the given rows of the stored points."""
    q = stored[torch.as_tensor(rows, device=stored.device)].cpu().numpy()
    if dtype == "f32":
        return q.astype(np.float64)
    if dtype == "bf16":
        return oracle.decode_bf16(q.view(np.uint16))
    s = scales[torch.as_tensor(rows, device=stored.device)].cpu().numpy().astype(np.float64)
    return oracle.decode_e4m3(q) * s[:, None]


def _store(x, dtype):
    if dtype == "f32":
        return x, None
    if dtype == "bf16":
        return kpp.quantize(x, "bf16"), None
    return kpp.quantize(x, "fp8")


@pytest.mark.parametrize("name,dtype,form", [
    ("gmm-N1e7-d64-K1024", "f32", kpp.FORM_PERSISTENT),
    ("gmm-N1e7-d64-K1024", "bf16", kpp.FORM_STREAMED),
    ("gmm-N2e7-d128-K2048-t3", "f32", kpp.FORM_PERSISTENT),
    ("gmm-N2e7-d128-K2048-t3", "bf16", kpp.FORM_PERSISTENT),
    ("gmm-N2e7-d128-K2048-t3", "fp8", kpp.FORM_STREAMED),
])
def test_full_size_sampled_parity(name, dtype, form):
    wl = datagen.WORKLOADS[name]
    N, d, K = wl.N, wl.d, wl.K
    x = datagen.workload_points(wl, DEV)
    stored, scales = _store(x, dtype)
    del x
    torch.cuda.empty_cache()
    opts = {"form": form}
    idx_t, d2_t, phi_t = kpp.seed(stored, K, SEED, dtype=dtype, row_scales=scales, opts=opts)
    idx = idx_t.cpu().numpy()
    d2 = d2_t.cpu().numpy()
    phi = float(phi_t.cpu()[0])

    # properties at any size
    assert np.all((idx >= 0) & (idx < N)) and len(np.unique(idx)) == K
    assert np.all(d2[idx] == 0.0) and np.all(d2 >= 0.0)
    s64 = d2.astype(np.float64).sum()
    assert abs(phi - s64) <= 1e-9 * s64
    # first seed
    assert idx[0] == min(int(oracle.uniform(SEED, 0, 0) * N), N - 1)

    # sampled D^2 against the FP64 minimum over all chosen centres
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(N, 2000, replace=False))
    xs = _decode(stored, scales, dtype, rows)
    cs = _decode(stored, scales, dtype, idx)
    best = np.full(rows.size, np.inf)
    for k0 in range(0, K, 128):
        diff = xs[:, None, :] - cs[None, k0:k0 + 128, :]
        best = np.minimum(best, np.einsum("ijk,ijk->ij", diff, diff).min(axis=1))
    got = d2[rows].astype(np.float64)
    zero = best == 0.0
    assert np.all(got[zero] == 0.0)
    rel = np.abs(got[~zero] - best[~zero]) / best[~zero]
    assert rel.max() <= 1e-5, rel.max()

    # sampled draws, replayed by the oracle's inverse CDF on the run's own D^2
    events = 0
    for m in (1, K // 2, K - 1):
        i_m, d2m_t, _ = kpp.seed(stored, m, SEED, dtype=dtype, row_scales=scales, opts=opts)
        assert np.array_equal(i_m.cpu().numpy(), idx[:m])  # same trajectory
        d2m = d2m_t.cpu().numpy().astype(np.float64)
        j, t, T = oracle.pick(d2m, oracle.uniform(SEED, 0, m))
        if j != idx[m]:
            lo, hi = sorted((j, int(idx[m])))
            P = np.cumsum(d2m[lo:hi])
            before = d2m[:lo].sum()
            # every prefix between the two choices within 1e-9 * T of t
            assert np.all(np.abs(before + P - t) <= 1e-9 * T), (m, j, idx[m])
            events += 1
    assert events <= 1


def _sharded(stored, K, world):
    """One point-sharded seeding of `stored` with `world` shards on this GPU
    (each shard's rows in an allocation of its own); returns numpy idx, D^2
    (all rows, in order) and phi."""
    from paper_1908_02136_gb300 import multi

    N = stored.shape[0]
    shards = [kpp.PointShard(stored[lo:hi].clone(), lo, N, K, SEED, 0, r, world)
              for r, (lo, hi) in enumerate(multi.shard_rows(N, world))]
    multi.seed_sharded(shards, multi.InProcessComm(), K)
    torch.cuda.synchronize()
    assert all(s.status() == kpp.OK for s in shards)
    idx = shards[0].idx.cpu().numpy()
    for s in shards[1:]:
        assert np.array_equal(s.idx.cpu().numpy(), idx)
    d2 = np.concatenate([s.d2.cpu().numpy() for s in shards])
    return idx, d2, float(shards[0].phi.cpu()[0])


@pytest.mark.parametrize("name,world", [("gmm-N1e7-d64-K1024", 3), ("gmm-N2e7-d128-K2048-t3", 2)])
def test_full_size_sharded_parity(name, world):
    """The point-sharded form at the full sizes, its shards on this GPU: the
    same sampled checks as the single-GPU forms above."""
    wl = datagen.WORKLOADS[name]
    N, d, K = wl.N, wl.d, wl.K
    x = datagen.workload_points(wl, DEV)
    idx, d2, phi = _sharded(x, K, world)
    assert np.all((idx >= 0) & (idx < N)) and len(np.unique(idx)) == K
    assert np.all(d2[idx] == 0.0) and np.all(d2 >= 0.0)
    s64 = d2.astype(np.float64).sum()
    assert abs(phi - s64) <= 1e-9 * s64
    assert idx[0] == min(int(oracle.uniform(SEED, 0, 0) * N), N - 1)
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(N, 2000, replace=False))
    xs = _decode(x, None, "f32", rows)
    cs = _decode(x, None, "f32", idx)
    best = np.full(rows.size, np.inf)
    for k0 in range(0, K, 128):
        diff = xs[:, None, :] - cs[None, k0:k0 + 128, :]
        best = np.minimum(best, np.einsum("ijk,ijk->ij", diff, diff).min(axis=1))
    got = d2[rows].astype(np.float64)
    zero = best == 0.0
    assert np.all(got[zero] == 0.0)
    assert (np.abs(got[~zero] - best[~zero]) / best[~zero]).max() <= 1e-5
    events = 0
    for m in (1, K // 2, K - 1):
        i_m, d2m, _ = _sharded(x, m, world)
        assert np.array_equal(i_m, idx[:m])  # same trajectory
        d2m = d2m.astype(np.float64)
        j, t, T = oracle.pick(d2m, oracle.uniform(SEED, 0, m))
        if j != idx[m]:
            lo, hi = sorted((j, int(idx[m])))
            P = np.cumsum(d2m[lo:hi])
            before = d2m[:lo].sum()
            assert np.all(np.abs(before + P - t) <= 1e-9 * T), (m, j, idx[m])
            events += 1
    assert events <= 1
