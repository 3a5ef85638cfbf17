"""GPU parity of k-means|| (kpp_kmeans_par, through the C ABI) against the
FP64 oracle:

* integer coordinates (|x| <= 64): every distance, sum and product is exact
  in the GPU's arithmetic, so the candidate list, the weights, D^2 after the
  rounds, each point's nearest candidate and the chosen centres must equal
  the oracle's end-to-end run bit for bit (duplicate points included, which
  exercises the earliest-candidate tie rule);
* Gaussian mixtures, replayed round by round: a run stopped after r rounds
  is the prefix of a longer run, the oracle's Bernoulli decisions on the
  GPU's own D^2 and phi reproduce round r's candidates exactly, D^2 is within
  1e-5 of the FP64 distance to the candidate each point holds, which is the
  FP64 nearest or a near tie within the tensor-core bound (counted), the
  weights are the histogram of those, and the oracle's weighted k-means++
  replayed on the GPU's candidates and weights draws the GPU's centres (or
  a counted near-boundary event);
* more than 4096 new candidates in a round (several tensor-core launches),
  rounds = 0, K = N, degenerate data, too small a candidate room, ragged N
  and d, determinism.
"""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _run(x_np, K, seed, rounds, ell, stream=0, cand_cap=None):
    x = torch.from_numpy(x_np).to(DEV)
    r = kpp.kmeans_par(x, K, seed, stream, ell=ell, rounds=rounds, cand_cap=cand_cap)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}


def _nearest(X, C):
    """FP64 nearest candidate (earliest on ties) and its distance."""
    best = np.full(X.shape[0], np.inf)
    arg = np.zeros(X.shape[0], dtype=np.int64)
    for k0 in range(0, C.shape[0], 256):
        diff = X[:, None, :] - C[None, k0:k0 + 256, :]
        dd = np.einsum("ijk,ijk->ij", diff, diff)
        j = dd.argmin(axis=1)
        v = dd[np.arange(X.shape[0]), j]
        better = v < best
        best = np.where(better, v, best)
        arg = np.where(better, j + k0, arg)
    return arg, best


@pytest.mark.parametrize("N,d,K,rounds,ell", [(3000, 2, 8, 3, 16.0), (5000, 32, 20, 4, 40.0),
                                              (4099, 65, 16, 5, 24.0), (777, 128, 5, 2, 10.0),
                                              (20000, 8, 64, 5, 128.0)])
def test_integer_regime_matches_oracle_exactly(N, d, K, rounds, ell):
    x = datagen.integer_points(N, d, seed=N + d, n_comp=8)
    seed, stream = 3, 1
    g = _run(x, K, seed, rounds, ell, stream)
    o = oracle.kmeans_par(x, K, ell, rounds, seed, stream)
    assert g["status"] == kpp.OK and o["status"] == 0
    assert np.array_equal(g["cand"], o["cand"])
    assert np.array_equal(g["weights"], o["w"])
    assert np.array_equal(g["idx"], o["idx"])
    D2, phi = oracle.min_update(x, o["cand"])
    assert np.array_equal(g["d2"].astype(np.float64), D2)
    assert g["phi"][0] == phi
    lab, _ = _nearest(x.astype(np.float64), x[o["cand"]].astype(np.float64))
    assert np.array_equal(g["labels"], lab)


def test_duplicates_in_one_round_take_the_earliest_candidate():
    # 40 distinct integer points, each repeated 50 times: a round can choose
    # several copies of one point, and all copies then belong to the first
    base = datagen.integer_points(40, 3, seed=5, n_comp=4)
    x = np.repeat(base, 50, axis=0)
    rng = np.random.default_rng(0)
    x = x[rng.permutation(x.shape[0])].copy()
    g = _run(x, 10, 7, 3, 200.0)
    o = oracle.kmeans_par(x, 10, 200.0, 3, 7, 0)
    assert np.array_equal(g["cand"], o["cand"])
    assert np.array_equal(g["weights"], o["w"])
    assert np.array_equal(g["idx"], o["idx"])
    assert g["status"] == o["status"] == 0


@pytest.mark.parametrize("N,d,K,ell", [(20000, 32, 32, 64.0), (12007, 64, 50, 100.0),
                                       (6000, 100, 16, 32.0)])
def test_float_regime_replayed_round_by_round(N, d, K, ell):
    rounds = 4
    x = datagen.gmm(N, d, K, seed=d)
    X = x.astype(np.float64)
    seed, stream = 11, 2
    runs = [_run(x, K, seed, r, ell, stream) for r in range(rounds + 1)]
    assert runs[0]["cand"][0] == min(int(oracle.uniform(seed, stream, 0) * N), N - 1)
    events = 0
    for r in range(rounds + 1):
        g = runs[r]
        cand = g["cand"]
        C = X[cand]
        # D^2 and the nearest candidate after r rounds
        lab = g["labels"].astype(np.int64)
        dist_g = ((X - C[lab]) ** 2).sum(1)
        nz = dist_g > 0
        assert np.all(g["d2"][~nz] == 0)
        assert np.max(np.abs(g["d2"][nz] - dist_g[nz]) / dist_g[nz]) <= 1e-5
        arg, best = _nearest(X, C)
        diff = lab != arg
        bound = (parity.LABEL_BOUND * np.linalg.norm(X, axis=1) * np.linalg.norm(C, axis=1).max()
                 + 1e-30)
        assert np.all(dist_g[diff] - best[diff] <= bound[diff])
        events += int(diff.sum())
        assert diff.sum() <= max(2, parity.LABEL_EVENT_FRAC * N)
        phi = float(g["phi"][0])
        assert phi == pytest.approx(g["d2"].astype(np.float64).sum(), rel=1e-12)
        assert np.array_equal(g["weights"], np.bincount(lab, minlength=cand.size))
        if r < rounds:
            nxt = runs[r + 1]["cand"]
            assert np.array_equal(nxt[:cand.size], cand)  # same trajectory
            flags, p, u = oracle.kmpar_select(g["d2"].astype(np.float64), phi, ell, seed, stream,
                                              r)
            assert np.array_equal(nxt[cand.size:], np.flatnonzero(flags))
    # the recluster replayed by the oracle on the GPU's candidates and weights
    g = runs[rounds]
    pos_of = {int(c): i for i, c in enumerate(g["cand"])}
    pos = np.array([pos_of[int(i)] for i in g["idx"]])
    _, own, st = oracle.weighted_seed(x, g["cand"], g["weights"], K, seed, stream, forced=pos)
    assert st == 0
    assert np.sum(own != pos) <= 1
    assert len(np.unique(g["idx"])) == K


def test_more_new_candidates_than_one_assignment_launch():
    # ell = N: every point with D^2 > 0 has p >= 1 at some rounds; round 0
    # alone appends thousands of candidates (several 4096-candidate chunks)
    N, d = 12000, 16
    x = datagen.integer_points(N, d, seed=2, n_comp=6)
    g = _run(x, 6, 1, 1, float(N) * 0.8, cand_cap=N)
    o = oracle.kmeans_par(x, 6, float(N) * 0.8, 1, 1, 0, cand_cap=N)
    assert g["cand"].size > 4096 + 1
    assert np.array_equal(g["cand"], o["cand"])
    assert np.array_equal(g["weights"], o["w"])
    assert np.array_equal(g["idx"], o["idx"])


def test_zero_rounds_and_k_equals_n():
    x = datagen.gmm(300, 4, 3, seed=1)
    g = _run(x, 1, 5, 0, 4.0)
    assert g["cand"].size == 1 and g["weights"][0] == 300 and g["idx"][0] == g["cand"][0]
    g = _run(x, 2, 5, 0, 4.0)
    assert g["status"] == kpp.ERR_DEGENERATE and g["idx"][1] == -1
    # K = N with ell large enough that every point becomes a candidate
    x = datagen.integer_points(64, 3, seed=3, n_comp=2)
    x = np.unique(x, axis=0)
    n = x.shape[0]
    g = _run(x, n, 9, 6, 1e9, cand_cap=n)
    o = oracle.kmeans_par(x, n, 1e9, 6, 9, 0, cand_cap=n)
    assert g["cand"].size == n
    assert np.array_equal(g["cand"], o["cand"]) and np.array_equal(g["idx"], o["idx"])
    assert g["status"] == kpp.OK


def test_degenerate_data():
    x = np.ones((500, 8), dtype=np.float32)
    g = _run(x, 1, 1, 3, 10.0)
    assert g["status"] == kpp.OK and g["cand"].size == 1 and float(g["phi"][0]) == 0.0
    g = _run(x, 3, 1, 3, 10.0)
    assert g["status"] == kpp.ERR_DEGENERATE


def test_capacity_and_argument_errors():
    x = torch.from_numpy(datagen.gmm(2000, 8, 4, seed=4)).to(DEV)
    with pytest.raises(kpp.KppError) as e:
        kpp.kmeans_par(x, 4, 1, rounds=3, ell=500.0, cand_cap=50)
    assert e.value.status == kpp.ERR_CAPACITY
    with pytest.raises(kpp.KppError) as e:
        kpp.kmeans_par(x, 4, 1, rounds=3, ell=-1.0)
    assert e.value.status == kpp.ERR_INVALID_ARG
    with pytest.raises(kpp.KppError) as e:
        kpp.kmeans_par(x, 2001, 1)
    assert e.value.status == kpp.ERR_INVALID_ARG
    small = torch.empty(256, dtype=torch.uint8, device=DEV)
    with pytest.raises(kpp.KppError) as e:
        kpp.kmeans_par(x, 4, 1, workspace=small)
    assert e.value.status == kpp.ERR_WORKSPACE


def test_deterministic():
    x = datagen.gmm(30000, 32, 16, seed=6)
    a = _run(x, 16, 4, 5, 32.0)
    b = _run(x, 16, 4, 5, 32.0)
    for k in ("cand", "weights", "idx", "labels", "d2", "phi"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.slow
def test_full_size_workload_sampled():
    """10^7 x 64, K = 1024, ell = 2K, 5 rounds (the k-means|| bench workload):
    the last round replayed exactly, D^2 of sampled rows against the FP64
    nearest candidate, weights, and the recluster replayed on the
    candidates' rows."""
    wl = datagen.WORKLOADS["gmm-N1e7-d64-K1024"]
    N, d, K = wl.N, wl.d, wl.K
    ell, seed, stream = 2.0 * K, wl.draw_seed, 0
    x = datagen.workload_points(wl, DEV)
    r4 = kpp.kmeans_par(x, K, seed, stream, ell=ell, rounds=4)
    r5 = kpp.kmeans_par(x, K, seed, stream, ell=ell, rounds=5)
    torch.cuda.synchronize()
    assert r5["status"] == kpp.OK
    c4, c5 = r4["cand"].cpu().numpy(), r5["cand"].cpu().numpy()
    assert c5[0] == min(int(oracle.uniform(seed, stream, 0) * N), N - 1)
    assert np.array_equal(c5[:c4.size], c4) and len(np.unique(c5)) == c5.size
    # the fifth round's Bernoulli decisions, replayed on the fourth's D^2 and phi
    flags, _, _ = oracle.kmpar_select(r4["d2"].cpu().numpy().astype(np.float64),
                                      float(r4["phi"].cpu()[0]), ell, seed, stream, 4)
    assert np.array_equal(c5[c4.size:], np.flatnonzero(flags))
    # weights: a histogram of the nearest candidates; every candidate holds itself
    w = r5["weights"].cpu().numpy()
    lab = r5["labels"].cpu().numpy()
    assert w.sum() == N and np.all(w >= 1)
    assert np.array_equal(lab[c5], np.arange(c5.size))
    # sampled D^2 against the FP64 nearest candidate
    rows = np.sort(np.random.default_rng(3).choice(N, 2000, replace=False))
    X = x[torch.as_tensor(rows, device=DEV)].cpu().numpy().astype(np.float64)
    C = x[r5["cand"]].cpu().numpy().astype(np.float64)
    arg, best = _nearest(X, C)
    d2 = r5["d2"].cpu().numpy()[rows].astype(np.float64)
    held = ((X - C[lab[rows]]) ** 2).sum(1)
    nz = held > 0  # a sampled row may be a candidate itself
    assert np.all(d2[~nz] == 0)
    assert np.max(np.abs(d2[nz] - held[nz]) / held[nz]) <= 1e-5
    bound = parity.LABEL_BOUND * np.linalg.norm(X, axis=1) * np.linalg.norm(C, axis=1).max()
    assert np.all(held - best <= bound)
    assert np.mean(lab[rows] != arg) <= max(2 / len(rows), parity.LABEL_EVENT_FRAC)
    # the recluster, replayed on the candidates' own rows
    idx = r5["idx"].cpu().numpy()
    pos_of = {int(c): i for i, c in enumerate(c5)}
    pos = np.array([pos_of[int(i)] for i in idx])
    _, own, st = oracle.weighted_seed(C.astype(np.float32), np.arange(c5.size), w, K, seed,
                                      stream, forced=pos)
    assert st == 0 and np.sum(own != pos) <= 1
