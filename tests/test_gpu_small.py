"""GPU parity of the small form (one CTA holding the points and D^2 in
shared memory for all K passes, through the C ABI) against the FP64 oracle:
bit-exact on integer coordinates, within 1e-5 relative D^2 and the draw band
otherwise, for every stored dtype, the specialised and the generic d, fewer
and more rows than threads, forced prefixes, degenerate data, K = 1, K = N,
N = 1, forced FP64 draw decisions, and the size limit."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SMALL = {"form": kpp.FORM_SMALL}


def _store(x_np, dtype):
    x = torch.from_numpy(x_np).to(DEV)
    if dtype == "f32":
        return x, None, x_np, None
    if dtype == "bf16":
        q = kpp.quantize(x, "bf16")
        return q, None, q.cpu().numpy().view(np.uint16), None
    q, s = kpp.quantize(x, "fp8")
    return q, s, q.cpu().numpy(), s.cpu().numpy()


def run(x_np, K, seed, dtype="f32", opts=SMALL, forced=None, check=True, stream_id=0):
    st, sc, st_np, sc_np = _store(x_np, dtype)
    idx, d2, phi = kpp.seed(st, K, seed, stream_id, dtype=dtype, row_scales=sc, opts=opts,
                            forced=forced, check=check)
    torch.cuda.synchronize()
    return st_np, sc_np, idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0])


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("N,d,K", [(10_000, 2, 16), (777, 4, 33), (3_001, 8, 40), (1_024, 16, 64),
                                   (5_000, 3, 25), (2_049, 5, 12), (12_000, 1, 30), (900, 31, 20)])
def test_small_integer_regime_bit_identical(N, d, K, dtype):
    x = datagen.integer_points(N, d, seed=N + d, n_comp=8)
    st, sc, idx, d2, phi = run(x, K, 17, dtype)
    parity.check(st, K, 17, 0, idx, d2, phi, exact=True)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("N,d,K", [(10_000, 2, 16), (4_000, 8, 40), (2_500, 16, 64),
                                   (6_000, 6, 30)])
def test_small_float_regime(N, d, K, dtype):
    x = datagen.gmm(N, d, K, seed=N + 2, mean_box=50.0)
    st, sc, idx, d2, phi = run(x, K, 5, dtype)
    assert parity.check(st, K, 5, 0, idx, d2, phi, scales=sc) <= 1


def test_small_paper_workload_is_the_automatic_choice():
    wl = datagen.WORKLOADS["gmm-N1e4-d2-K16"]
    x = datagen.workload_points(wl)
    st, plan = kpp.kpp_describe(wl.N, wl.d, wl.K, kpp.F32)
    assert st == kpp.OK and plan.form == kpp.FORM_SMALL and plan.grid == 1
    a = run(x, wl.K, wl.draw_seed, opts=None)
    assert parity.check(a[0], wl.K, wl.draw_seed, 0, a[2], a[3], a[4]) == 0
    b = run(x, wl.K, wl.draw_seed, opts={"form": kpp.FORM_PERSISTENT})
    assert np.array_equal(a[2], b[2])  # same draws as the persistent form


def test_small_forced_prefix_and_exact_draws():
    x = datagen.gmm(8_000, 4, 16, seed=6)
    r = oracle.seed(x, 20, 4)
    st, sc, idx, d2, phi = run(x, 20, 4, forced=r["idx"])
    assert np.array_equal(idx, r["idx"])
    np.testing.assert_allclose(d2, r["d2"], rtol=1e-5)
    st, sc, idx2, d2b, phi2 = run(x, 20, 4, forced=r["idx"][:7])
    assert np.array_equal(idx2[:7], r["idx"][:7])
    parity.check(st, 20, 4, 0, idx2, d2b, phi2)
    a = run(x, 20, 4, opts=dict(SMALL, exact_draws=1))
    b = run(x, 20, 4)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3]) and a[4] == b[4]
    xi = datagen.integer_points(5_000, 8, seed=3, n_comp=8)  # 180 KB: fits
    st, sc, idx, d2, phi = run(xi, 40, 2, opts=dict(SMALL, exact_draws=1))
    parity.check(st, 40, 2, 0, idx, d2, phi, exact=True)


def test_small_edge_cases():
    x = datagen.gmm(257, 4, 4, seed=8)
    st, sc, idx, d2, phi = run(x, 1, 2)
    parity.check(st, 1, 2, 0, idx, d2, phi)
    st, sc, idx, d2, phi = run(x, 257, 2)
    assert sorted(idx.tolist()) == list(range(257)) and np.all(d2 == 0) and phi == 0.0
    st, sc, idx, d2, phi = run(np.array([[1.5, -2.0]], np.float32), 1, 0)
    assert idx.tolist() == [0] and d2.tolist() == [0.0] and phi == 0.0
    # more passes than draws computed ahead at once (1024)
    xi = datagen.integer_points(3_000, 2, seed=1, lo=-1400, hi=1400)  # D^2 < 2^24
    st, sc, idx, d2, phi = run(xi, 1_500, 9)
    parity.check(st, 1_500, 9, 0, idx, d2, phi, exact=True)


def test_small_degenerate_data_and_bad_forced_index():
    base = np.array([[0, 0, 0, 0], [1, 2, 3, 4], [5, 5, 5, 5]], np.float32)
    x = np.repeat(base, [400, 300, 301], axis=0)
    x = x[np.random.default_rng(0).permutation(len(x))]
    with pytest.raises(kpp.KppError) as e:
        run(x, 5, 1)
    assert e.value.status == kpp.ERR_DEGENERATE
    st, sc, idx, d2, phi = run(x, 5, 1, check=False)
    assert np.all(idx[3:] == -1) and phi == 0.0
    parity.check(st, 5, 1, 0, idx, d2, phi, exact=True, status=oracle.DEGENERATE)
    y = torch.zeros((64, 4), device=DEV)
    y[:, 0] = torch.arange(64, device=DEV, dtype=torch.float32)
    for forced in ([5, 64], [-1]):
        with pytest.raises(kpp.KppError) as e:
            kpp.seed(y, 3, 1, forced=forced, opts=SMALL)
        assert e.value.status == kpp.ERR_INVALID_ARG


def test_small_size_limit():
    # 60 000 x 3 FP32 points plus D^2 need 960 KB: more than one SM holds
    st, plan = kpp.kpp_describe(60_000, 3, 8, kpp.F32, SMALL)
    assert st == kpp.ERR_UNSUPPORTED
    st, plan = kpp.kpp_describe(60_000, 3, 8, kpp.F32)
    assert st == kpp.OK and plan.form != kpp.FORM_SMALL
    # a FP32 d = 2 problem near the limit, seeded exactly
    N = 17_500
    xi = datagen.integer_points(N, 2, seed=5, n_comp=8)
    st, plan = kpp.kpp_describe(N, 2, 24, kpp.F32, SMALL)
    assert st == kpp.OK and plan.smem_bytes == 12 * N
    s, sc, idx, d2, phi = run(xi, 24, 3)
    parity.check(s, 24, 3, 0, idx, d2, phi, exact=True)
