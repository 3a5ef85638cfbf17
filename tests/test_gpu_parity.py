"""GPU parity of the streamed seeding path (through the C ABI) against the FP64
oracle: bit-exact in the integer regime, within 1e-5 relative D^2 and the
near-boundary draw band in the float regime, for every stored dtype, ragged
sizes, the generic kernel, every lanes-per-row specialisation, graph and
plain launches, degenerate data and forced prefixes."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
STREAMED, PERSISTENT = kpp.FORM_STREAMED, kpp.FORM_PERSISTENT
FORMS = [STREAMED, PERSISTENT]


def run(points_np, K, seed, stream_id=0, *, dtype="f32", opts=None, forced=None, check=True):
    """Stores the points as `dtype` on the GPU (quantising with the library)
    and seeds; returns numpy (stored points, scales, idx, d2, phi)."""
    x = torch.from_numpy(points_np).to(DEV)
    scales = None
    if dtype == "f32":
        stored = x
        stored_np = points_np
    elif dtype == "bf16":
        stored = kpp.quantize(x, "bf16")
        stored_np = stored.cpu().numpy().view(np.uint16)
    else:
        stored, scales = kpp.quantize(x, "fp8")
        stored_np = stored.cpu().numpy()
    idx, d2, phi = kpp.seed(stored, K, seed, stream_id, dtype=dtype, row_scales=scales,
                            opts=opts, forced=forced, check=check)
    torch.cuda.synchronize()
    sc = None if scales is None else scales.cpu().numpy()
    return stored_np, sc, idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0])


EXACT_SHAPES = [(5000, 2, 16), (7777, 4, 33), (4097, 8, 40), (20011, 16, 64), (20011, 32, 64),
                (3001, 64, 20), (4099, 128, 12), (1000, 3, 10), (999, 5, 9), (2500, 96, 8)]


def _form_ok(form, d):
    # the persistent form is built for d in {2,4,...,128}; others use the streamed form
    return form == STREAMED or d in (2, 4, 8, 16, 32, 64, 128)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("N,d,K", EXACT_SHAPES)
def test_exact_regime_bit_identical(N, d, K, dtype, form):
    x = datagen.integer_points(N, d, seed=N + d, n_comp=8)
    if not _form_ok(form, d):
        with pytest.raises(kpp.KppError) as e:
            run(x, K, seed=17, dtype=dtype, opts={"form": form})
        assert e.value.status == kpp.ERR_UNSUPPORTED
        return
    # small blocks so that even these sizes span several CTAs
    opts = {"form": form, "min_rows_per_cta": 256}
    st, sc, idx, d2, phi = run(x, K, seed=17, dtype=dtype, opts=opts)
    parity.check(st, K, 17, 0, idx, d2, phi, scales=sc, exact=True)


@pytest.mark.parametrize("N,d,K,ncomp", [(10_000, 2, 16, 16), (100_003, 32, 64, 64),
                                         (50_001, 64, 48, 32), (30_011, 128, 32, 32),
                                         (12_345, 8, 100, 50), (9_999, 7, 20, 10)])
@pytest.mark.parametrize("form", FORMS)
def test_float_regime_f32(N, d, K, ncomp, form):
    x = datagen.gmm(N, d, ncomp, seed=N, mean_box=50.0)
    if not _form_ok(form, d):
        return
    st, sc, idx, d2, phi = run(x, K, seed=1, opts={"form": form, "min_rows_per_cta": 512})
    events = parity.check(st, K, 1, 0, idx, d2, phi)
    assert events <= 1


@pytest.mark.parametrize("form", FORMS)
def test_paper_scale_small_workload(form):
    wl = datagen.WORKLOADS["gmm-N1e4-d2-K16"]
    x = datagen.workload_points(wl)
    st, sc, idx, d2, phi = run(x, wl.K, seed=wl.draw_seed, opts={"form": form})
    assert parity.check(st, wl.K, wl.draw_seed, 0, idx, d2, phi) == 0


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("N,d,K", [(40_003, 16, 32), (20_001, 64, 24), (10_007, 128, 16),
                                   (8_191, 2, 12), (6_001, 4, 12), (5_003, 8, 10)])
@pytest.mark.parametrize("form", FORMS)
def test_float_regime_low_precision_storage(N, d, K, dtype, form):
    x = datagen.gmm(N, d, K, seed=N + 1, mean_box=50.0)
    st, sc, idx, d2, phi = run(x, K, seed=5, dtype=dtype,
                               opts={"form": form, "min_rows_per_cta": 1024})
    events = parity.check(st, K, 5, 0, idx, d2, phi, scales=sc)
    assert events <= 1


@pytest.mark.parametrize("d,lanes", [(8, 1), (8, 2), (16, 2), (16, 4), (32, 2), (32, 4),
                                     (32, 8), (64, 4), (64, 8), (64, 16), (128, 8), (128, 16),
                                     (128, 32)])
def test_every_lanes_per_row_variant(d, lanes):
    x = datagen.integer_points(9001, d, seed=d * lanes, n_comp=6)
    opts = {"lanes_per_row": lanes, "form": STREAMED}
    st, sc, idx, d2, phi = run(x, 24, seed=3, opts=opts)
    parity.check(st, 24, 3, 0, idx, d2, phi, exact=True)


def test_unbuilt_lanes_variant_is_rejected():
    x = torch.zeros((100, 32), device=DEV)
    for form in FORMS:
        with pytest.raises(kpp.KppError) as e:
            kpp.seed(x, 4, 1, opts={"lanes_per_row": 32, "form": form})
        assert e.value.status == kpp.ERR_UNSUPPORTED


def test_graph_and_plain_launches_agree_and_repeat():
    x = datagen.gmm(60_000, 32, 32, seed=2)
    a = run(x, 40, seed=9, opts={"form": STREAMED})
    b = run(x, 40, seed=9, opts={"use_graph": -1, "form": STREAMED})
    c = run(x, 40, seed=9, opts={"form": STREAMED})  # graph cache hit
    for other in (b, c):
        assert np.array_equal(a[2], other[2])
        assert np.array_equal(a[3], other[3])
        assert a[4] == other[4]


def test_blocking_changes_nothing_in_exact_regime():
    x = datagen.integer_points(50_000, 16, seed=4, n_comp=8)
    ref = run(x, 30, seed=4, opts={"form": STREAMED})
    variants = [{"form": STREAMED, "ctas_per_sm": c} for c in (1, 2, 3)]
    variants += [{"form": PERSISTENT, "min_rows_per_cta": r} for r in (256, 1000, 5000, 60_000)]
    variants += [{"form": PERSISTENT, "ctas_per_sm": 2, "min_rows_per_cta": 128}]
    for o in variants:
        v = run(x, 30, seed=4, opts=o)
        assert np.array_equal(ref[2], v[2]) and np.array_equal(ref[3], v[3]), o
        assert ref[4] == v[4], o


@pytest.mark.parametrize("opts", [
    {"smem_cache": -1}, {"smem_cache": 0}, {"smem_cache": 1024}, {"alternate": -1},
    {"alternate": 1}, {"l2_policy": -1}, {"l2_policy": 2}, {"l2_policy": 0},
    # D^2 too large for shared memory: kept in the output array
    {"min_rows_per_cta": 70_000, "smem_cache": -1},
    {"min_rows_per_cta": 70_000, "smem_cache": 0},
])
def test_persistent_options_exact(opts):
    x = datagen.integer_points(150_001, 8, seed=12, n_comp=16)
    o = dict(opts, form=PERSISTENT)
    o.setdefault("min_rows_per_cta", 2048)
    st, sc, idx, d2, phi = run(x, 40, seed=21, opts=o)
    parity.check(st, 40, 21, 0, idx, d2, phi, exact=True)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_persistent_d2_in_global_float(dtype):
    x = datagen.gmm(200_003, 32, 64, seed=13)
    o = {"form": PERSISTENT, "min_rows_per_cta": 70_000}
    st, sc, idx, d2, phi = run(x, 48, seed=2, dtype=dtype, opts=o)
    assert parity.check(st, 48, 2, 0, idx, d2, phi, scales=sc) <= 1


def test_barrier_timeout_is_reported_not_hung():
    # A 1 us bound on every grid-barrier wait cannot hold across 64 passes over
    # 10^6 points: some CTA gives up, records the timeout and every CTA exits.
    x = torch.from_numpy(datagen.gmm(1_000_000, 32, 32, seed=3)).to(DEV)
    with pytest.raises(kpp.KppError) as e:
        kpp.seed(x, 64, 1, opts={"form": PERSISTENT, "timeout_us": 1})
    assert e.value.status == kpp.ERR_TIMEOUT
    # the context is still usable and a normal call succeeds afterwards
    idx, d2, phi = kpp.seed(x, 64, 1, opts={"form": PERSISTENT})
    assert int((idx >= 0).sum()) == 64


@pytest.mark.parametrize("form", FORMS)
def test_k1_and_k_equals_n(form):
    x = datagen.gmm(257, 4, 4, seed=8)
    st, sc, idx, d2, phi = run(x, 1, seed=2, opts={"form": form})
    parity.check(st, 1, 2, 0, idx, d2, phi)
    st, sc, idx, d2, phi = run(x, 257, seed=2, opts={"form": form})
    assert sorted(idx.tolist()) == list(range(257))
    assert np.all(d2 == 0) and phi == 0.0


@pytest.mark.parametrize("form", FORMS)
def test_single_point(form):
    x = np.array([[1.5, -2.0]], np.float32)
    st, sc, idx, d2, phi = run(x, 1, seed=0, opts={"form": form})
    assert idx.tolist() == [0] and d2.tolist() == [0.0] and phi == 0.0


@pytest.mark.parametrize("form", FORMS)
def test_degenerate_data_reports_status(form):
    base = np.array([[0, 0, 0, 0], [1, 2, 3, 4], [5, 5, 5, 5]], np.float32)
    x = np.repeat(base, [400, 300, 301], axis=0)
    rng = np.random.default_rng(0)
    x = x[rng.permutation(len(x))]
    o = {"form": form, "min_rows_per_cta": 128}
    with pytest.raises(kpp.KppError) as e:
        run(x, 5, seed=1, opts=o)
    assert e.value.status == kpp.ERR_DEGENERATE
    st, sc, idx, d2, phi = run(x, 5, seed=1, check=False, opts=o)
    assert np.all(idx[3:] == -1) and phi == 0.0
    parity.check(st, 5, 1, 0, idx, d2, phi, exact=True, status=oracle.DEGENERATE)


@pytest.mark.parametrize("form", FORMS)
def test_forced_prefix_replays_the_oracle(form):
    x = datagen.gmm(30_000, 16, 16, seed=6)
    r = oracle.seed(x, 20, 4)
    o = {"form": form, "min_rows_per_cta": 1024}
    st, sc, idx, d2, phi = run(x, 20, seed=4, forced=r["idx"], opts=o)
    assert np.array_equal(idx, r["idx"])
    np.testing.assert_allclose(d2, r["d2"], rtol=1e-5)
    # a partial prefix: the GPU continues with its own draws after it
    st, sc, idx2, d2, phi = run(x, 20, seed=4, forced=r["idx"][:7], opts=o)
    assert np.array_equal(idx2[:7], r["idx"][:7])
    parity.check(st, 20, 4, 0, idx2, d2, phi)


@pytest.mark.parametrize("form", FORMS)
def test_bad_forced_index_is_a_device_error(form):
    x = torch.zeros((64, 4), device=DEV)
    x[:, 0] = torch.arange(64, device=DEV, dtype=torch.float32)
    for forced in ([5, 64], [-1], [3, 7, 1 << 40]):
        with pytest.raises(kpp.KppError) as e:
            kpp.seed(x, 3, 1, forced=forced, opts={"form": form})
        assert e.value.status == kpp.ERR_INVALID_ARG


def test_streams_give_independent_draws():
    x = datagen.gmm(20_000, 8, 16, seed=9)
    a = run(x, 16, seed=1, stream_id=0)
    b = run(x, 16, seed=1, stream_id=1)
    assert not np.array_equal(a[2], b[2])
    parity.check(b[0], 16, 1, 1, b[2], b[3], b[4])


def test_quantizers_match_the_oracle_bit_for_bit():
    x = datagen.gmm(33_333, 24, 8, seed=3, mean_box=80.0)
    x[5] = 0.0
    xt = torch.from_numpy(x).to(DEV)
    qb = kpp.quantize(xt, "bf16").cpu().numpy().view(np.uint16)
    assert np.array_equal(qb, oracle.quantize_bf16(x))
    q8, s8 = kpp.quantize(xt, "fp8")
    oq, os_ = oracle.quantize_fp8(x)
    assert np.array_equal(s8.cpu().numpy(), os_)
    assert np.array_equal(q8.cpu().numpy(), oq)
    # odd element count for the BF16 tail
    y = x.ravel()[:1001].reshape(1001, 1).copy()
    qy = kpp.quantize(torch.from_numpy(y).to(DEV), "bf16").cpu().numpy().view(np.uint16)
    assert np.array_equal(qy, oracle.quantize_bf16(y))


def test_seed_host_matches_device_seed():
    x = datagen.gmm(70_001, 32, 32, seed=11)
    st, sc, idx, d2, phi = run(x, 32, seed=2)
    xh = torch.from_numpy(x).pin_memory()
    hidx, hd2, hphi, status, _ = kpp.seed_host(xh, 32, 2)
    assert status == kpp.OK
    assert np.array_equal(hidx.numpy(), idx)
    assert np.array_equal(hd2.numpy(), d2)
    assert float(hphi[0]) == phi


@pytest.mark.slow
@pytest.mark.parametrize("form", FORMS)
def test_full_size_workload_parity(form):
    """The bench workload (10^6 x 32, K=256) in the bench's launch configuration
    (the persistent form with default options is what bench.py times)."""
    wl = datagen.WORKLOADS["gmm-N1e6-d32-K256"]
    x = datagen.workload_points(wl)
    st, sc, idx, d2, phi = run(x, wl.K, seed=wl.draw_seed, opts={"form": form})
    events = parity.check(st, wl.K, wl.draw_seed, 0, idx, d2, phi)
    assert events <= 2


def test_random_shapes_sweep():
    """Seeded random shapes in the exact (integer) regime: N log-uniform in
    [1, 200 000], d from specialised and generic widths, K up to 300, random
    draw seed and stream, random CTA block sizes; per shape two random
    (form, storage) pairs among auto / streamed / persistent / small and
    FP32 / BF16, each bit-identical to the oracle (a form that cannot take
    the shape must say so with KPP_ERR_UNSUPPORTED)."""
    rng = np.random.default_rng(7)
    dims = [1, 2, 3, 4, 5, 7, 8, 16, 17, 32, 33, 64, 100, 128]
    forms = [kpp.FORM_AUTO, STREAMED, PERSISTENT, kpp.FORM_SMALL]
    for case in range(24):
        N = int(round(np.exp(rng.uniform(0.0, np.log(200_000)))))
        d = int(rng.choice(dims))
        K = int(rng.integers(1, min(N, 300) + 1))
        seed, sid = int(rng.integers(1, 1 << 30)), int(rng.integers(0, 1000))
        x = datagen.integer_points(N, d, seed=case, n_comp=int(rng.integers(1, 9)))
        for _ in range(2):
            form = int(rng.choice(forms))
            dtype = str(rng.choice(["f32", "bf16"]))
            opts = {"form": form, "min_rows_per_cta": int(rng.choice([0, 128, 1024]))}
            try:
                st, sc, idx, d2, phi = run(x, K, seed=seed, stream_id=sid, dtype=dtype, opts=opts)
            except kpp.KppError as e:
                assert e.status == kpp.ERR_UNSUPPORTED and form != kpp.FORM_AUTO, (N, d, K, form)
                continue
            parity.check(st, K, seed, sid, idx, d2, phi, scales=sc, exact=True)
