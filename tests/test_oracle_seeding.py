"""Pins for the oracle's seeding loop (Algorithm 1 of arXiv:1908.02136 with
readings R1-R6): distances against scipy, the draw against numpy's
searchsorted on a cumulative sum, the invariants of the method, replay of a
forced prefix and the degenerate stop."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

from paper_1908_02136_gb300 import datagen


def test_k1_is_uniform_pick_and_exact_sqeuclidean(oracle_mod):
    x = datagen.gmm(500, 7, 4, seed=3, mean_box=10.0)
    for s in range(5):
        r = oracle_mod.seed(x, 1, seed=s)
        i0 = int(np.floor(oracle_mod.uniform(s, 0, 0) * 500))
        assert r["idx"].tolist() == [i0]
        ref = cdist(x.astype(np.float64), x[i0:i0 + 1].astype(np.float64), "sqeuclidean")[:, 0]
        np.testing.assert_allclose(r["d2"], ref, rtol=1e-13, atol=0)
        assert r["phi"] == pytest.approx(ref.sum(), rel=1e-13)


def test_d2_is_min_over_chosen_centres(oracle_mod):
    x = datagen.gmm(2000, 5, 8, seed=4, mean_box=20.0)
    r = oracle_mod.seed(x, 12, seed=9, history=True)
    xd = x.astype(np.float64)
    for m in range(12):
        ref = cdist(xd, xd[r["idx"][:m + 1]], "sqeuclidean").min(axis=1)
        np.testing.assert_allclose(r["d2_hist"][m], ref, rtol=1e-12, atol=1e-9)


def test_pick_is_inverse_cdf(oracle_mod):
    rng = np.random.default_rng(2)
    for trial in range(300):
        n = int(rng.integers(1, 60))
        d2 = rng.exponential(size=n) * (rng.random(n) < 0.7)
        u = rng.random()
        i, t, T = oracle_mod.pick(d2, u)
        if d2.sum() == 0:
            assert i == -1
            continue
        cum = np.cumsum(d2)
        ref = int(np.searchsorted(cum, u * cum[-1], side="right"))
        if ref >= n:  # rounding left no prefix above t: largest positive weight
            ref = int(np.nonzero(d2 > 0)[0][-1])
        assert i == ref and d2[i] > 0


def test_pick_edge_cases(oracle_mod):
    # u = 0 draws the first positive weight; a zero-weight point is never drawn.
    assert oracle_mod.pick(np.array([0.0, 0.0, 2.0, 1.0]), 0.0)[0] == 2
    assert oracle_mod.pick(np.array([1.0, 0.0, 1.0]), 0.5)[0] == 2
    assert oracle_mod.pick(np.array([1.0, 0.0, 1.0]), 0.49)[0] == 0
    # u just below 1 draws the last positive weight
    assert oracle_mod.pick(np.array([1.0, 3.0, 0.0]), np.nextafter(1.0, 0.0))[0] == 1
    assert oracle_mod.pick(np.zeros(5), 0.3)[0] == -1


def test_invariants_on_distinct_points(oracle_mod):
    x = datagen.gmm(3000, 3, 10, seed=5, mean_box=10.0)
    assert len(np.unique(x, axis=0)) == len(x)
    r = oracle_mod.seed(x, 40, seed=11, history=True)
    idx, hist = r["idx"], r["d2_hist"]
    assert len(set(idx.tolist())) == 40  # no repeated index
    assert np.all(np.diff(hist, axis=0) <= 0)  # D^2 non-increasing per point
    for m in range(40):
        assert np.all(hist[m:, idx[m]] == 0.0)  # a chosen point has D^2 = 0 exactly
    assert r["phi"] == pytest.approx(hist[-1].sum(), rel=1e-14)


def test_k_equals_n_is_a_permutation(oracle_mod):
    x = datagen.gmm(64, 2, 4, seed=6, mean_box=5.0)
    r = oracle_mod.seed(x, 64, seed=1)
    assert sorted(r["idx"].tolist()) == list(range(64))
    assert r["phi"] == 0.0 and np.all(r["d2"] == 0.0)


def test_duplicates_and_degenerate_stop(oracle_mod):
    base = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]], np.float32)
    x = np.repeat(base, [5, 3, 4], axis=0)
    r = oracle_mod.seed(x, 6, seed=2)
    assert r["status"] == oracle_mod.DEGENERATE
    idx = r["idx"]
    assert np.all(idx[3:] == -1)
    assert len({tuple(x[i]) for i in idx[:3]}) == 3  # one seed per distinct value
    assert r["phi"] == 0.0
    # exactly as many seeds as distinct values: no degenerate stop
    r = oracle_mod.seed(x, 3, seed=2)
    assert r["status"] == oracle_mod.OK and r["phi"] == 0.0


def test_forced_replay_reproduces_and_reports(oracle_mod):
    x = datagen.gmm(4000, 8, 16, seed=7, mean_box=10.0)
    r = oracle_mod.seed(x, 20, seed=3, draws=True)
    rep = oracle_mod.seed(x, 20, seed=3, forced=r["idx"], draws=True)
    assert np.array_equal(rep["idx"], r["idx"]) and np.array_equal(rep["d2"], r["d2"])
    dr = rep["draws"]
    assert np.array_equal(dr["own"][1:], r["idx"][1:])
    for m in range(1, 20):
        assert dr["P_before"][m] <= dr["t"][m] < dr["P_at"][m]
    # A different forced prefix changes the trajectory after it, and the oracle
    # reports its own would-be draw at every step.
    forced = r["idx"].copy()
    forced[5] = (forced[5] + 1) % 4000
    rep2 = oracle_mod.seed(x, 20, seed=3, forced=forced[:6], draws=True)
    assert np.array_equal(rep2["idx"][:6], forced[:6])
    assert rep2["draws"]["own"][5] == r["idx"][5]


def test_bf16_and_fp8_points_are_decoded_exactly(oracle_mod):
    import torch

    x = datagen.gmm(800, 16, 8, seed=8, mean_box=30.0)
    qb = oracle_mod.quantize_bf16(x)
    xb = torch.from_numpy(qb.view(np.int16)).view(torch.bfloat16).double().numpy()
    rb = oracle_mod.seed(qb, 6, seed=4)
    ref = cdist(xb, xb[rb["idx"]], "sqeuclidean").min(axis=1)
    np.testing.assert_allclose(rb["d2"], ref, rtol=1e-12, atol=1e-9)
    q8, s8 = oracle_mod.quantize_fp8(x)
    x8 = torch.from_numpy(q8).view(torch.float8_e4m3fn).double().numpy() * s8[:, None]
    r8 = oracle_mod.seed(q8, 6, seed=4, scales=s8)
    ref = cdist(x8, x8[r8["idx"]], "sqeuclidean").min(axis=1)
    np.testing.assert_allclose(r8["d2"], ref, rtol=1e-12, atol=1e-9)


def test_invalid_arguments_are_rejected(oracle_mod):
    x = np.zeros((4, 2), np.float32)
    with pytest.raises(ValueError):
        oracle_mod.seed(x, 5, seed=0)  # K > N
    with pytest.raises(ValueError):
        oracle_mod.seed(x, 2, seed=0, forced=np.array([7]))
    with pytest.raises(ValueError):
        oracle_mod.seed(np.zeros((4, 2), np.uint8), 2, seed=0)  # FP8 without scales
