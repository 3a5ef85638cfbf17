"""The multi-threaded FP64 oracle (the CPU baseline on all host cores)
against the serial oracle, which the other oracle tests pin to the paper's
Algorithm 1.  Per-point arithmetic is the same, so D^2 must be bit-identical;
the draw's prefix sums are regrouped at chunk boundaries, which changes
nothing on integer data (every sum exact) and at most the last bits of phi
on mixtures."""
import numpy as np
import pytest

from paper_1908_02136_gb300 import datagen


@pytest.mark.parametrize("threads", [1, 2, 3, 7, 16])
@pytest.mark.parametrize("N,d,K", [(20_011, 16, 40), (4_099, 128, 12), (9_999, 3, 25),
                                   (1_000, 2, 64)])
def test_mt_bit_identical_on_integer_data(oracle_mod, N, d, K, threads):
    x = datagen.integer_points(N, d, seed=N + d, n_comp=8)
    a = oracle_mod.seed(x, K, 17)
    b = oracle_mod.seed_mt(x, K, 17, threads=threads)
    assert b["status"] == a["status"] == oracle_mod.OK
    assert np.array_equal(a["idx"], b["idx"])
    assert np.array_equal(a["d2"], b["d2"])
    assert a["phi"] == b["phi"]


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_mt_bit_identical_stored_formats_integer_data(oracle_mod, dtype):
    x = datagen.integer_points(30_001, 32, seed=5, n_comp=8)
    if dtype == "bf16":
        st, sc = oracle_mod.quantize_bf16(x), None
    else:
        st, sc = oracle_mod.quantize_fp8(x)
    a = oracle_mod.seed(st, 24, 3, scales=sc)
    b = oracle_mod.seed_mt(st, 24, 3, scales=sc, threads=5)
    assert np.array_equal(a["idx"], b["idx"])
    assert np.array_equal(a["d2"], b["d2"])
    if dtype == "bf16":
        assert a["phi"] == b["phi"]
    else:
        assert abs(a["phi"] - b["phi"]) <= 1e-12 * a["phi"]


@pytest.mark.parametrize("threads", [2, 5, 8])
def test_mt_matches_serial_on_mixtures(oracle_mod, threads):
    wl = datagen.WORKLOADS["gmm-N1e4-d2-K16"]
    for x, K in [(datagen.workload_points(wl), wl.K),
                 (datagen.gmm(150_000, 32, 64, seed=2), 64)]:
        a = oracle_mod.seed(x, K, 1)
        b = oracle_mod.seed_mt(x, K, 1, threads=threads)
        assert np.array_equal(a["idx"], b["idx"])
        assert np.array_equal(a["d2"], b["d2"])
        assert abs(a["phi"] - b["phi"]) <= 1e-12 * a["phi"]


def test_mt_edge_cases(oracle_mod):
    x = datagen.gmm(37, 4, 4, seed=8)
    # more threads than points, K = N: a permutation with phi = 0
    b = oracle_mod.seed_mt(x, 37, 2, threads=64)
    assert sorted(b["idx"].tolist()) == list(range(37)) and b["phi"] == 0.0
    assert b["threads"] == 37
    # K = 1: the uniform first pick and D^2 to it
    a = oracle_mod.seed(x, 1, 9)
    b = oracle_mod.seed_mt(x, 1, 9, threads=4)
    assert np.array_equal(a["idx"], b["idx"]) and np.array_equal(a["d2"], b["d2"])
    # degenerate data stops the same way (reading R4)
    base = np.array([[0, 0], [1, 2], [5, 5]], np.float32)
    y = np.repeat(base, [40, 30, 31], axis=0)
    a = oracle_mod.seed(y, 5, 1)
    b = oracle_mod.seed_mt(y, 5, 1, threads=3)
    assert a["status"] == b["status"] == oracle_mod.DEGENERATE
    assert np.array_equal(a["idx"], b["idx"])
    with pytest.raises(ValueError):
        oracle_mod.seed_mt(x, 38, 1)
