"""Pins for the oracle's sampling law: the D^2 weighting of k-means++
(Algorithm 1 of arXiv:1908.02136) checked against exact enumeration of the
probability tree on tiny inputs, a hand-derived golden table, and the
expected-cost bound E[phi] <= 8 (ln K + 2) phi_opt of Arthur and
Vassilvitskii (the paper's reference [2])."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sqdist(a, b):
    return sum((Fraction(int(p)) - Fraction(int(q))) ** 2 for p, q in zip(a, b))


def exact_sequences(X, K):
    """{ordered index tuple: (exact probability, exact phi)} for integer points.

    Enumerates the k-means++ tree: uniform first seed, then each next seed with
    probability D^2 / sum D^2; a zero total stops the sequence (padded by -1).
    """
    N = len(X)
    out = {}

    def rec(seq, d2, prob):
        if len(seq) == K:
            out[tuple(seq)] = (prob, sum(d2))
            return
        T = sum(d2)
        if T == 0:
            out[tuple(seq + [-1] * (K - len(seq)))] = (prob, Fraction(0))
            return
        for j in range(N):
            if d2[j] > 0:
                nd = [min(d2[i], _sqdist(X[i], X[j])) for i in range(N)]
                rec(seq + [j], nd, prob * d2[j] / T)

    for i0 in range(N):
        d2 = [_sqdist(X[i], X[i0]) for i in range(N)]
        rec([i0], d2, Fraction(1, N))
    return out


def _chi2(oracle_mod, X, K, n_seeds, stream=0):
    table = exact_sequences(X, K)
    pts = np.asarray(X, dtype=np.float32)
    counts = {}
    for s in range(n_seeds):
        seq = tuple(oracle_mod.seed(pts, K, seed=s, stream=stream)["idx"].tolist())
        counts[seq] = counts.get(seq, 0) + 1
    assert set(counts) <= set(table), set(counts) - set(table)
    keys = sorted(table, key=lambda k: -table[k][0])
    exp = np.array([float(table[k][0]) * n_seeds for k in keys])
    obs = np.array([counts.get(k, 0) for k in keys], dtype=float)
    # merge bins with expected count below 5 into one
    small = exp < 5
    if small.any():
        exp = np.append(exp[~small], exp[small].sum())
        obs = np.append(obs[~small], obs[small].sum())
    return stats.chisquare(obs, exp).pvalue, table, counts


CASES = [
    # (points, K)
    ([[0], [1], [3], [7]], 2),
    ([[0], [1], [3], [7], [8], [20]], 3),
    ([[0, 0], [2, 0], [0, 3], [5, 5], [1, 1]], 3),
    ([[0, 0], [0, 0], [4, 1], [1, 4], [9, 9], [3, 3]], 3),  # a duplicate pair
    ([[0, 0], [0, 0], [0, 0], [1, 1]], 3),  # degenerate: 2 distinct points, K=3
]


def _alt_law(X, K, power):
    """Sequence probabilities when seeds are drawn proportional to D^power."""
    X = np.asarray(X, dtype=np.float64)
    N = len(X)
    D = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    out = {}

    def rec(seq, d2, prob):
        if len(seq) == K:
            out[tuple(seq)] = prob
            return
        w = d2 ** (power / 2.0)
        if w.sum() == 0:
            out[tuple(seq + [-1] * (K - len(seq)))] = prob
            return
        for j in range(N):
            if w[j] > 0:
                rec(seq + [j], np.minimum(d2, D[j]), prob * w[j] / w.sum())

    for i0 in range(N):
        rec([i0], D[i0].copy(), 1.0 / N)
    return out


@pytest.mark.parametrize("X,K", CASES)
def test_sampling_law_chi_square(oracle_mod, X, K):
    n = 100_000
    p, table, counts = _chi2(oracle_mod, X, K, n)
    assert p > 1e-4, p
    # The same counts reject plausible wrong laws (weights D or D^4 instead of
    # D^2), so the test has the power to catch a dropped or doubled square.
    for power in (1, 4):
        alt = _alt_law(X, K, power)
        if all(abs(alt.get(k, 0.0) - float(v[0])) < 1e-3 for k, v in table.items()):
            continue  # laws coincide on this input (e.g. all distances 0 or 1)
        keys = sorted(set(alt) | set(counts))
        exp = np.array([alt.get(k, 0.0) * n for k in keys])
        obs = np.array([counts.get(k, 0) for k in keys], dtype=float)
        if np.any((exp == 0) & (obs > 0)):
            continue  # impossible under the wrong law: rejected outright
        keep = exp >= 5
        exp_m = np.append(exp[keep], exp[~keep].sum())
        obs_m = np.append(obs[keep], obs[~keep].sum())
        if exp_m[-1] == 0:
            exp_m, obs_m = exp_m[:-1], obs_m[:-1]
        exp_m *= obs_m.sum() / exp_m.sum()
        assert stats.chisquare(obs_m, exp_m).pvalue < 1e-6, power


def test_sampling_law_other_stream(oracle_mod):
    p, _, _ = _chi2(oracle_mod, [[0], [2], [3], [9], [10]], 3, 50_000, stream=77)
    assert p > 1e-4, p


def test_golden_hand_derived_pairs(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "tiny_1d_k2.json")))
    X = [[v] for v in g["points_1d"]]
    table = exact_sequences(X, g["K"])
    for key, frac in g["pair_probabilities"].items():
        i0, i1 = map(int, key.split(","))
        assert table[(i0, i1)][0] == Fraction(frac)
        assert table[(i0, i1)][1] == g["pair_phi"][key]
    assert sum(v[0] for v in table.values()) == 1
    e_phi = sum(Fraction(t) for t in g["expected_phi_terms"])
    assert sum(p * f for p, f in table.values()) == e_phi
    # Monte-Carlo mean of the oracle's phi agrees with the exact expectation.
    pts = np.asarray(X, dtype=np.float32)
    phis = np.array([oracle_mod.seed(pts, 2, seed=s)["phi"] for s in range(40_000)])
    se = phis.std() / math.sqrt(len(phis))
    assert abs(phis.mean() - float(e_phi)) < 5 * se


def _phi_opt(X, K):
    """Optimal k-means cost by brute force over all K^N labelings."""
    X = np.asarray(X, dtype=np.float64)
    best = math.inf
    for lab in itertools.product(range(K), repeat=len(X)):
        lab = np.array(lab)
        cost = 0.0
        for k in range(K):
            pts = X[lab == k]
            if len(pts):
                cost += ((pts - pts.mean(0)) ** 2).sum()
        best = min(best, cost)
    return best


@pytest.mark.parametrize("X,K", [
    ([[0], [1], [3], [7]], 2),
    ([[0, 0], [1, 0], [0, 1], [10, 10], [11, 10], [10, 11], [-9, 8], [-8, 8]], 3),
    ([[0], [1], [2], [50], [51], [100], [101], [102]], 3),
])
def test_expected_cost_bound(oracle_mod, X, K):
    g = json.load(open(os.path.join(GOLDEN, "tiny_1d_k2.json")))
    table = exact_sequences(X, K)
    e_phi = float(sum(p * f for p, f in table.values()))
    opt = _phi_opt(X, K)
    if X == [[v] for v in g["points_1d"]]:
        assert opt == pytest.approx(float(Fraction(g["phi_opt"])))
    assert e_phi <= 8 * (math.log(K) + 2) * opt
    # and the oracle's own mean cost matches the exact expectation
    pts = np.asarray(X, dtype=np.float32)
    phis = np.array([oracle_mod.seed(pts, K, seed=s)["phi"] for s in range(20_000)])
    se = phis.std() / math.sqrt(len(phis))
    assert abs(phis.mean() - e_phi) < 5 * se + 1e-12
