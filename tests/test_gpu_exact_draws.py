"""The draw's exact FP64 decision path, forced on every comparison.

A draw decides "prefix P > t" (t = u * T, the draw's point on the cumulative
D^2 of Algorithm 1's probability line) from an FP32 estimate of P - t, and
falls back to the exact FP64 comparison only when the estimate lies within
2^-40 t of t.  Random draws almost never land in that band, so the fallback
would otherwise go untested.  With ``exact_draws`` every comparison -- block,
warp segment, 32-row chunk or sub-slice, point -- takes the fallback, in the
persistent, streamed and batched forms.

Two things must hold:
* integer coordinates (every D^2, prefix and total exact): indices, D^2 and
  phi bit-identical to the FP64 oracle;
* any data: indices, D^2 and phi identical to the default path's, since the
  FP32 estimate only ever decides where the exact answer is certain.
"""
import numpy as np
import pytest
import torch

import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
STREAMED, PERSISTENT = kpp.FORM_STREAMED, kpp.FORM_PERSISTENT


def _store(x_np, dtype):
    x = torch.from_numpy(x_np).to(DEV)
    if dtype == "f32":
        return x, None, x_np
    if dtype == "bf16":
        q = kpp.quantize(x, "bf16")
        return q, None, q.cpu().numpy().view(np.uint16)
    q, s = kpp.quantize(x, "fp8")
    return q, s, q.cpu().numpy()


def _seed(stored, scales, K, seed, dtype, opts):
    idx, d2, phi = kpp.seed(stored, K, seed, dtype=dtype, row_scales=scales, opts=opts)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0])


# (options of the form) -- small row blocks so that every level of the draw
# has several candidates; the last two keep D^2 in the output array, where
# the persistent form's owner searches sub-slices instead of 32-row chunks
FORM_OPTS = [
    {"form": STREAMED},
    {"form": STREAMED, "ctas_per_sm": 1},
    {"form": PERSISTENT, "min_rows_per_cta": 256},
    {"form": PERSISTENT, "min_rows_per_cta": 2048},
    {"form": PERSISTENT, "min_rows_per_cta": 70_000, "smem_cache": -1},
]


@pytest.mark.parametrize("opts", FORM_OPTS)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("N,d,K", [(20_011, 16, 64), (150_001, 8, 40), (4_099, 128, 12),
                                   (7_777, 4, 33)])
def test_exact_decisions_integer_regime(N, d, K, dtype, opts):
    x = datagen.integer_points(N, d, seed=N + d, n_comp=8)
    stored, scales, stored_np = _store(x, dtype)
    ex = _seed(stored, scales, K, 17, dtype, dict(opts, exact_draws=1))
    parity.check(stored_np, K, 17, 0, *ex, exact=True)
    df = _seed(stored, scales, K, 17, dtype, opts)
    assert np.array_equal(ex[0], df[0]) and np.array_equal(ex[1], df[1]) and ex[2] == df[2]


@pytest.mark.parametrize("opts", FORM_OPTS)
@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_exact_decisions_float_regime(dtype, opts):
    x = datagen.gmm(120_007, 32, 48, seed=5, mean_box=50.0)
    stored, scales, stored_np = _store(x, dtype)
    ex = _seed(stored, scales, 48, 3, dtype, dict(opts, exact_draws=1))
    assert parity.check(stored_np, 48, 3, 0, *ex, scales=None if scales is None
                        else scales.cpu().numpy()) <= 1
    df = _seed(stored, scales, 48, 3, dtype, opts)
    assert np.array_equal(ex[0], df[0]) and np.array_equal(ex[1], df[1]) and ex[2] == df[2]


@pytest.mark.parametrize("exact", [True, False])
def test_exact_decisions_batched(exact):
    rng = np.random.default_rng(3)
    probs = []
    for i in range(24):
        N = int(rng.integers(500, 90_000))
        d = int(rng.choice([2, 8, 16, 32, 64, 128]))
        K = int(rng.integers(2, min(48, N)))
        x = (datagen.integer_points(N, d, seed=300 + i, n_comp=6) if exact
             else datagen.gmm(N, d, K, seed=300 + i))
        probs.append((x, K))
    xs = [torch.from_numpy(x).to(DEV) for x, _ in probs]
    Ks = [K for _, K in probs]
    sids = list(range(len(probs)))
    outs_ex, _ = kpp.seed_batched(xs, Ks, [1] * len(xs), sids, opts={"exact_draws": 1})
    outs_df, _ = kpp.seed_batched(xs, Ks, [1] * len(xs), sids)
    torch.cuda.synchronize()
    for (x, K), sid, a, b in zip(probs, sids, outs_ex, outs_df):
        ia, da, pa = a[0].cpu().numpy(), a[1].cpu().numpy(), float(a[2].cpu()[0])
        ib, db, pb = b[0].cpu().numpy(), b[1].cpu().numpy(), float(b[2].cpu()[0])
        assert np.array_equal(ia, ib) and np.array_equal(da, db) and pa == pb
        events = parity.check(x, K, 1, sid, ia, da, pa, exact=exact)
        assert events <= 1
