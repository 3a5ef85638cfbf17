"""Pins of the oracle's Lloyd iteration (readings L1-L3) against libraries
and facts other than itself: scipy's vector quantisation for the
assignment, scikit-learn's one-iteration Lloyd for the new centres, the
monotone decrease of the k-means cost, tie and empty-cluster rules, and the
decoded precision forms."""
import numpy as np
import pytest
from scipy.cluster.vq import vq
from scipy.spatial.distance import cdist

import oracle
from paper_1908_02136_gb300 import datagen


def _data(N=400, d=5, K=6, seed=0):
    x = datagen.gmm(N, d, K, seed=seed)
    rng = np.random.default_rng(seed + 1)
    C = x[rng.choice(N, K, replace=False)].astype(np.float64)
    return x, C


def test_assignment_matches_scipy_vq():
    for seed in range(5):
        x, C = _data(seed=seed)
        r = oracle.lloyd_step(x, C)
        code, dist = vq(x.astype(np.float64), C)
        assert np.array_equal(r["labels"], code.astype(np.int32))
        np.testing.assert_allclose(np.sqrt(r["d2"]), dist, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r["d2"], cdist(x.astype(np.float64), C, "sqeuclidean").min(1),
                                   rtol=1e-12)
        assert r["phi"] == pytest.approx(r["d2"].sum(), rel=1e-12)


def test_new_centres_match_sklearn_one_lloyd_iteration():
    KMeans = pytest.importorskip("sklearn.cluster").KMeans
    for seed in range(3):
        x, C = _data(N=600, d=4, K=5, seed=10 + seed)
        r = oracle.lloyd_step(x, C)
        assert np.all(r["counts"] > 0)  # sklearn relocates empty clusters
        km = KMeans(n_clusters=C.shape[0], init=C, n_init=1, max_iter=1, tol=0.0,
                    algorithm="lloyd").fit(x.astype(np.float64))
        np.testing.assert_allclose(r["centres"], km.cluster_centers_, rtol=1e-10, atol=1e-10)
        assert np.array_equal(np.bincount(r["labels"], minlength=C.shape[0]), r["counts"])


def test_cost_never_increases():
    x, C = _data(N=800, d=3, K=7, seed=4)
    phis = []
    for _ in range(12):
        r = oracle.lloyd_step(x, C)
        phis.append(r["phi"])
        C = r["centres"]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(phis, phis[1:]))
    assert phis[-1] < phis[0]


def test_ties_go_to_the_smallest_index_and_empty_clusters_stay():
    x = np.array([[0.0, 0.0], [2.0, 0.0], [1.0, 0.0], [10.0, 0.0]], np.float32)
    C = np.array([[2.0, 0.0], [0.0, 0.0], [50.0, 50.0]])
    r = oracle.lloyd_step(x, C)
    # point (1,0) is at distance 1 from centres 0 and 1: centre 0 wins
    assert list(r["labels"]) == [1, 0, 0, 0]
    assert list(r["counts"]) == [3, 1, 0]
    np.testing.assert_array_equal(r["centres"][2], C[2])          # empty: unchanged
    np.testing.assert_allclose(r["centres"][0], [13.0 / 3.0, 0.0])  # (2 + 1 + 10) / 3
    np.testing.assert_allclose(r["centres"][1], [0.0, 0.0])
    assert r["phi"] == pytest.approx(0 + 0 + 1 + 64)


def test_precision_forms_use_the_decoded_values():
    x, C = _data(N=300, d=8, K=4, seed=7)
    q = oracle.quantize_bf16(x)
    dec = oracle.decode_bf16(q)
    r = oracle.lloyd_step(q, C, dtype="bf16")
    code, _ = vq(dec, C)
    assert np.array_equal(r["labels"], code.astype(np.int32))
    q8, s8 = oracle.quantize_fp8(x)
    dec8 = oracle.decode_e4m3(q8) * s8.astype(np.float64)[:, None]
    r8 = oracle.lloyd_step(q8, C, dtype="fp8", scales=s8)
    code8, _ = vq(dec8, C)
    assert np.array_equal(r8["labels"], code8.astype(np.int32))
    counts = np.bincount(code8, minlength=4)
    for k in range(4):
        if counts[k]:
            np.testing.assert_allclose(r8["centres"][k], dec8[code8 == k].mean(0), rtol=1e-12)
