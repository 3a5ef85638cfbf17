"""Pins of the oracle's k-means|| (readings P1-P4) against facts other than
itself: numpy's Philox4x64-10 at arbitrary counters, scipy's distances and
vector quantisation, the Bernoulli law of the oversampling (expected counts
and per-point frequencies), the exact weighted D^2 law of the recluster by
enumeration, its invariance to scaling the weights by a power of two, and
end-to-end properties on well-separated clusters."""
import itertools
from fractions import Fraction

import numpy as np
import pytest
from scipy.cluster.vq import vq
from scipy.spatial.distance import cdist
from scipy.stats import chisquare

import oracle
from paper_1908_02136_gb300 import datagen


def test_uniform_ctr_matches_numpy_philox():
    rng = np.random.default_rng(5)
    for _ in range(50):
        key = [int(v) for v in rng.integers(0, 2**63, size=2)]
        ctr = [int(v) for v in rng.integers(0, 2**63, size=4)]
        bg = np.random.Philox(counter=ctr, key=key)
        # numpy advances the counter by one before its first output block
        c = ctr[:]
        c[0] = (c[0] - 1) % 2**64
        bg2 = np.random.Philox(counter=c, key=key)
        w0 = int(bg2.random_raw(1)[0])
        u = oracle.uniform_ctr(key[0], key[1], *ctr)
        assert u == (w0 >> 11) * 2.0**-53
    # counter {m, 0, 0, 0} is the seeding draw
    for m in range(10):
        assert oracle.uniform_ctr(7, 3, m) == oracle.uniform(7, 3, m)


def test_min_update_matches_cdist():
    x = datagen.gmm(500, 6, 5, seed=2)
    c1, c2 = [3, 77], [150, 400, 401]
    D, phi = oracle.min_update(x, c1)
    ref = cdist(x.astype(np.float64), x[c1].astype(np.float64), "sqeuclidean").min(1)
    np.testing.assert_allclose(D, ref, rtol=1e-12, atol=1e-12)
    assert phi == pytest.approx(ref.sum(), rel=1e-12)
    D2, _ = oracle.min_update(x, c2, D)
    ref2 = cdist(x.astype(np.float64), x[c1 + c2].astype(np.float64), "sqeuclidean").min(1)
    np.testing.assert_allclose(D2, ref2, rtol=1e-12, atol=1e-12)


def test_oversampling_follows_the_bernoulli_law():
    # expected number selected = sum min(1, p); per-point frequencies = p
    D = np.array([0.0, 1.0, 2.0, 4.0, 8.0, 16.0, 100.0])
    phi = D.sum()
    ell = 3.0
    p = np.minimum(1.0, ell * D / phi)
    R = 20000
    hits = np.zeros(D.size)
    for s in range(R):
        f, pp, u = oracle.kmpar_select(D, phi, ell, seed=s, stream=1, r=s % 5)
        np.testing.assert_allclose(pp, ell * D / phi, rtol=0, atol=0)
        assert np.array_equal(f, (u < pp).astype(np.uint8))
        hits += f
    assert hits[0] == 0                       # D^2 = 0: never selected
    assert hits[-1] == R                      # p >= 1: always selected
    sd = np.sqrt(R * p * (1 - p)) + 1e-9
    assert np.all(np.abs(hits - R * p) <= 5 * sd)


def test_weights_match_scipy_vq():
    x = datagen.gmm(800, 3, 6, seed=3)
    cand = np.array([5, 17, 300, 301, 650, 799])
    w = oracle.kmpar_weights(x, cand)
    code, _ = vq(x.astype(np.float64), x[cand].astype(np.float64))
    assert np.array_equal(w, np.bincount(code, minlength=cand.size))
    assert w.sum() == 800


def _weighted_law(pts, w, K):
    """Exact probability of every ordered sequence of weighted D^2 draws."""
    n = len(pts)
    probs = {}
    for seq in itertools.permutations(range(n), K):
        pr = Fraction(w[seq[0]], sum(w))
        D = [None] * n
        for m in range(1, K):
            for c in range(n):
                dd = Fraction((pts[c] - pts[seq[m - 1]]) ** 2)
                D[c] = dd if D[c] is None or dd < D[c] else D[c]
            tot = sum(w[c] * D[c] for c in range(n))
            if tot == 0:
                pr = Fraction(0)
                break
            pr *= Fraction(w[seq[m]]) * D[seq[m]] / tot
        if pr:
            probs[seq] = pr
    return probs


def test_recluster_follows_the_weighted_d2_law():
    pts1 = [0, 1, 3, 7]
    w = [3, 1, 2, 1]
    x = np.array(pts1, dtype=np.float32)[:, None]
    cand = np.arange(4)
    K = 2
    law = _weighted_law([Fraction(v) for v in pts1], w, K)
    assert sum(law.values()) == 1
    R = 60000
    counts = {}
    for s in range(R):
        pos, own, st = oracle.weighted_seed(x, cand, w, K, seed=s, stream=2)
        assert st == oracle.OK
        counts[tuple(pos)] = counts.get(tuple(pos), 0) + 1
    seqs = sorted(law)
    obs = np.array([counts.get(q, 0) for q in seqs])
    exp = np.array([float(law[q]) * R for q in seqs])
    assert obs.sum() == R
    assert chisquare(obs, exp).pvalue > 1e-4


def test_recluster_is_invariant_to_power_of_two_weight_scaling():
    x = datagen.gmm(300, 5, 4, seed=4)
    cand = np.arange(0, 300, 7)
    w = np.random.default_rng(1).integers(1, 20, size=cand.size)
    for s in range(20):
        a, _, _ = oracle.weighted_seed(x, cand, w, 6, seed=s)
        b, _, _ = oracle.weighted_seed(x, cand, w * 8, 6, seed=s)
        assert np.array_equal(a, b)


def test_kmeans_par_covers_well_separated_clusters():
    # 6 tight, far-apart blobs: the chosen centres land one per blob
    rng = np.random.default_rng(9)
    means = np.arange(6)[:, None] * 1000.0 * np.ones((1, 3))
    lab = rng.integers(0, 6, size=1200)
    x = (means[lab] + rng.normal(size=(1200, 3))).astype(np.float32)
    covered = 0
    for s in range(20):
        r = oracle.kmeans_par(x, 6, ell=12.0, rounds=5, seed=s)
        assert r["status"] == oracle.OK
        assert len(set(r["idx"].tolist())) == 6
        assert r["w"].sum() == 1200 and r["cand"][0] == min(int(oracle.uniform(s, 0, 0) * 1200), 1199)
        assert np.all(np.diff(r["cand"][1:]) != 0)
        covered += len(set(lab[r["idx"]].tolist())) == 6
    assert covered >= 18


def test_kmeans_par_is_its_steps_in_order():
    # the end-to-end run against its steps wired here from the readings: P1
    # first seed and D^2, P2 round r drawn at counter {i, r + 1} with the
    # candidates appended in index order and D^2 / phi updated, P3 weights,
    # P4 the weighted recluster at counters {m, 0, 1, 0}
    x = datagen.gmm(700, 4, 5, seed=12)
    K, ell, rounds, seed, stream = 5, 9.0, 4, 21, 3
    r = oracle.kmeans_par(x, K, ell, rounds, seed, stream)
    N = x.shape[0]
    c0 = min(int(oracle.uniform(seed, stream, 0) * N), N - 1)
    cand = [c0]
    D2, phi = oracle.min_update(x, [c0])
    for rr in range(rounds):
        flags, p, u = oracle.kmpar_select(D2, phi, ell, seed, stream, rr)
        # the draws are Philox at counter {i, r + 1, 0, 0}
        for i in (0, N // 2, N - 1):
            assert u[i] == oracle.uniform_ctr(seed, stream, i, rr + 1, 0, 0)
        new = np.flatnonzero(flags)
        cand.extend(new.tolist())
        if new.size:
            D2, phi = oracle.min_update(x, new, D2)
    assert np.array_equal(r["cand"], np.array(cand))
    w = oracle.kmpar_weights(x, cand)
    assert np.array_equal(r["w"], w)
    pos, own, st = oracle.weighted_seed(x, cand, w, K, seed, stream)
    assert st == 0
    assert np.array_equal(r["idx"], np.array(cand)[pos])
