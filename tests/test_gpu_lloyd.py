"""GPU parity of one Lloyd iteration (kpp_lloyd_step, through the C ABI)
against the FP64 oracle's Lloyd step:

* integer coordinates (|x| <= 64): the split BF16 operands are exact, so the
  tensor-core scores are exact and labels, D^2, counts and the cost must be
  bit-identical to the oracle, centres equal to its FP64 means rounded once;
* Gaussian mixtures: every label is the oracle's or within the near-tie
  bound 2^-15 |x| max|c| of it (derived below; the events are counted and
  recorded as test properties), D^2 within 1e-5 of the FP64 distance to
  the chosen centre, centres within 1e-5 of the FP64 means of the GPU's own
  assignment, the cost within 1e-5;
* ragged N (not a multiple of the 128-point tile, fewer points than one
  tile), K across centre tiles and a partial last tile, d below, at and
  between the 64-feature chunks, empty clusters, several iterations, and
  argument errors.
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


def _step(x_np, C_np):
    x = torch.from_numpy(x_np).to(DEV)
    ll = kpp.Lloyd(x, C_np.shape[0])
    lab, d2, C2, cnt, phi = ll.step(torch.from_numpy(C_np.astype(np.float32)))
    torch.cuda.synchronize()
    return (lab.cpu().numpy(), d2.cpu().numpy(), C2.cpu().numpy(), cnt.cpu().numpy(),
            float(phi.cpu()[0]))


LABEL_BOUND, MAX_EVENT_FRAC = parity.LABEL_BOUND, parity.LABEL_EVENT_FRAC


def _check_float(x_np, C_np, record=None):
    lab, d2, C2, cnt, phi = _step(x_np, C_np)
    C64 = C_np.astype(np.float32).astype(np.float64)
    ref = oracle.lloyd_step(x_np, C64)
    X = x_np.astype(np.float64)
    N = X.shape[0]
    # every label is the oracle's, or a near tie within the bound
    dist_g = ((X - C64[lab]) ** 2).sum(1)
    dist_o = ref["d2"]
    diff = lab != ref["labels"]
    scale = np.linalg.norm(X, axis=1) * np.linalg.norm(C64, axis=1).max() + 1e-30
    gap = (dist_g[diff] - dist_o[diff]) / scale[diff]
    if record is not None:
        record("label_events", int(diff.sum()))
        record("max_gap_over_x_cmax", float(gap.max()) if gap.size else 0.0)
    assert np.all(gap <= LABEL_BOUND), gap.max()
    assert diff.sum() <= max(2, MAX_EVENT_FRAC * N), diff.sum()
    # D^2: FP32 difference form to the chosen centre
    nz = dist_g > 0
    assert np.all(d2[~nz] == 0)
    assert np.max(np.abs(d2[nz] - dist_g[nz]) / dist_g[nz]) <= 1e-5
    # counts and centres from the GPU's own assignment
    K = C64.shape[0]
    assert np.array_equal(cnt, np.bincount(lab, minlength=K))
    sums = np.zeros_like(C64)
    np.add.at(sums, lab, X)
    means = np.where(cnt[:, None] > 0, sums / np.maximum(cnt, 1)[:, None], C64)
    # per-CTA sums are FP32 (a few hundred points each), totals FP64
    np.testing.assert_allclose(C2, means, rtol=1e-5, atol=1e-5 * np.abs(means).max())
    assert phi == pytest.approx(dist_g.sum(), rel=1e-5)
    return diff.sum()


@pytest.mark.parametrize("N,d,K", [(1000, 8, 7), (5000, 64, 256), (4999, 128, 300),
                                   (127, 16, 5), (20000, 100, 1000), (3000, 2, 1)])
def test_integer_regime_bit_identical(N, d, K):
    x = datagen.integer_points(N, d, seed=N + d, n_comp=8)
    C = x[np.random.default_rng(K).choice(N, K, replace=False)].astype(np.float64)
    lab, d2, C2, cnt, phi = _step(x, C)
    ref = oracle.lloyd_step(x, C)
    assert np.array_equal(lab, ref["labels"])
    # the assignment entry point alone gives the same labels
    ll = kpp.Lloyd(torch.from_numpy(x).to(DEV), K)
    assert np.array_equal(ll.assign(torch.from_numpy(C.astype(np.float32))).cpu().numpy(), lab)
    assert np.array_equal(d2.astype(np.float64), ref["d2"])
    assert np.array_equal(cnt, ref["counts"])
    assert phi == ref["phi"]
    assert np.array_equal(C2, ref["centres"].astype(np.float32))


@pytest.mark.parametrize("N,d,K", [(20000, 32, 64), (30011, 64, 512), (10000, 128, 257),
                                   (8000, 48, 40)])
def test_float_regime(N, d, K, record_property):
    x = datagen.gmm(N, d, K, seed=d)
    C = x[np.random.default_rng(1).choice(N, K, replace=False)].astype(np.float64)
    _check_float(x, C, record_property)


def test_empty_clusters_keep_their_centre():
    x = datagen.gmm(3000, 16, 4, seed=3)
    C = np.concatenate([x[:4].astype(np.float64), np.full((3, 16), 1e4)])
    lab, d2, C2, cnt, phi = _step(x, C)
    assert np.all(cnt[4:] == 0)
    assert np.array_equal(C2[4:], C[4:].astype(np.float32))


def test_iterations_lower_the_cost():
    x_np = datagen.gmm(50_000, 32, 32, seed=9)
    x = torch.from_numpy(x_np).to(DEV)
    idx, _, _ = kpp.seed(x, 32, 1)
    C = x[idx]
    ll = kpp.Lloyd(x, 32)
    phis = []
    for _ in range(6):
        lab, d2, C, cnt, phi = ll.step(C)
        phis.append(float(phi.cpu()[0]))
    assert all(b <= a * (1 + 1e-6) for a, b in zip(phis, phis[1:]))
    assert phis[-1] < phis[0]


def test_argument_errors():
    x = torch.zeros((100, 200), device=DEV)
    with pytest.raises(kpp.KppError) as e:
        kpp.Lloyd(x, 4)
    assert e.value.status == kpp.ERR_INVALID_ARG
    assert kpp.kpp_lloyd_workspace_size(100, 8, 5000) == 0
    assert kpp.kpp_lloyd_workspace_size(10, 8, 11) == 0
    x = torch.zeros((100, 8), device=DEV)
    ll = kpp.Lloyd(x, 4)
    small = torch.empty(256, dtype=torch.uint8, device=DEV)
    c = torch.zeros((4, 8), device=DEV)
    lab = torch.empty(100, dtype=torch.int32, device=DEV)
    with torch.cuda.device(DEV):
        st = kpp.kpp_lloyd_step(x.data_ptr(), 100, 8, c.data_ptr(), 4, lab.data_ptr(), None,
                                torch.empty_like(c).data_ptr(), None, None, small.data_ptr(),
                                small.numel(), None)
    assert st == kpp.ERR_WORKSPACE


@pytest.mark.parametrize("N,d,K", [(127, 16, 5), (1000, 8, 7), (200_003, 32, 1000),
                                   (150_000, 128, 300), (100_000, 64, 4096), (70_001, 100, 257)])
def test_pair_and_single_sm_forms_agree(N, d, K, monkeypatch):
    """The CTA-pair assignment (256 x 256 MMAs over two SMs, the default)
    and the one-SM kernel add the same products per score in the same
    order, so their labels are identical: float data, ragged N (a pair whose
    second CTA has no points), K over partial and many centre tiles, both
    feature chunks, and N large enough that every cluster reuses its point
    buffers and centre stages."""
    x_np = datagen.gmm(N, d, min(K, 64), seed=N % 97)
    C = torch.from_numpy(x_np[np.random.default_rng(2).choice(N, K, replace=False)]).to(DEV)
    ll = kpp.Lloyd(torch.from_numpy(x_np).to(DEV), K)
    monkeypatch.setenv("KPP_LLOYD_PAIR", "0")
    single = ll.assign(C).cpu().numpy()
    monkeypatch.setenv("KPP_LLOYD_PAIR", "1")
    pair = ll.assign(C).cpu().numpy()
    assert np.array_equal(pair, single)
    # and the pair form against the oracle on a sample of points
    rows = np.random.default_rng(3).choice(N, min(N, 2000), replace=False)
    C64 = C.cpu().numpy().astype(np.float64)
    ref = oracle.lloyd_step(x_np[rows], C64)
    X = x_np[rows].astype(np.float64)
    dist_g = ((X - C64[pair[rows]]) ** 2).sum(1)
    diff = pair[rows] != ref["labels"]
    scale = np.linalg.norm(X, axis=1) * np.linalg.norm(C64, axis=1).max() + 1e-30
    assert np.all((dist_g[diff] - ref["d2"][diff]) / scale[diff] <= LABEL_BOUND)
    assert diff.sum() <= max(2, MAX_EVENT_FRAC * rows.size)


def test_pair_form_integer_regime_bit_identical(monkeypatch):
    """Integer coordinates over many groups per cluster: the pair form's
    labels equal the oracle's exactly."""
    monkeypatch.setenv("KPP_LLOYD_PAIR", "1")
    N, d, K = 300_000, 48, 700
    x = datagen.integer_points(N, d, seed=5, n_comp=16)
    C = x[np.random.default_rng(4).choice(N, K, replace=False)].astype(np.float64)
    lab, d2, C2, cnt, phi = _step(x, C)
    ref = oracle.lloyd_step(x, C)
    assert np.array_equal(lab, ref["labels"])
    assert np.array_equal(cnt, ref["counts"])


@pytest.mark.parametrize("pair", ["0", "1"])
def test_exact_ties_take_the_smallest_centre_index(pair, monkeypatch):
    """Integer points and centres with exact duplicates placed in the same
    32-column block, in different blocks of one tile and in different
    centre tiles (both kernels' tile widths): every label is the smallest
    index among the tied nearest centres, as in the oracle."""
    monkeypatch.setenv("KPP_LLOYD_PAIR", pair)
    N, d, K = 20_000, 24, 700
    x = datagen.integer_points(N, d, seed=11, n_comp=8)
    rng = np.random.default_rng(12)
    C = x[rng.choice(N, K, replace=False)].astype(np.float64)
    for src, dups in [(3, (17, 40)), (5, (130, 300, 520)), (200, (201, 699)), (257, (0,))]:
        for j in dups:
            C[j] = C[src]
    lab, d2, C2, cnt, phi = _step(x, C)
    ref = oracle.lloyd_step(x, C)
    assert np.array_equal(lab, ref["labels"])
    # the tie rule itself, independently of the oracle
    D = ((x[:, None, :].astype(np.float64) - C[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(lab, D.argmin(1))


def test_random_shapes_sweep(monkeypatch, record_property):
    """Seeded random shapes (N from 1 to 60 000, d from 1 to 128, K from 1
    to min(N, 4096)): the two assignment kernels give identical labels, and
    on integer coordinates both equal the oracle's; on float data every
    differing label is a near tie within the bound."""
    rng = np.random.default_rng(2024)
    events = []
    for case in range(14):
        N = int(rng.integers(1, 60_001)) if case else 1
        d = int(rng.integers(1, 129))
        K = int(rng.integers(1, min(N, 4096) + 1))
        integer = case % 2 == 0
        if integer:
            x = datagen.integer_points(N, d, seed=case, n_comp=min(K, 16))
        else:
            x = datagen.gmm(N, d, max(1, min(K, 32)), seed=case)
        C = x[rng.choice(N, K, replace=False)].astype(np.float64)
        ll = kpp.Lloyd(torch.from_numpy(x).to(DEV), K)
        Ct = torch.from_numpy(C.astype(np.float32)).to(DEV)
        monkeypatch.setenv("KPP_LLOYD_PAIR", "0")
        single = ll.assign(Ct).cpu().numpy()
        monkeypatch.setenv("KPP_LLOYD_PAIR", "1")
        pair = ll.assign(Ct).cpu().numpy()
        assert np.array_equal(pair, single), (N, d, K)
        rows = np.arange(N) if N <= 3000 else rng.choice(N, 3000, replace=False)
        ref = oracle.lloyd_step(x[rows], C)
        if integer:
            assert np.array_equal(pair[rows], ref["labels"]), (N, d, K)
        else:
            X = x[rows].astype(np.float64)
            dist_g = ((X - C[pair[rows]]) ** 2).sum(1)
            diff = pair[rows] != ref["labels"]
            scale = np.linalg.norm(X, axis=1) * np.linalg.norm(C, axis=1).max() + 1e-30
            assert np.all((dist_g[diff] - ref["d2"][diff]) / scale[diff] <= LABEL_BOUND), (N, d, K)
            # random centres can be dense (hundreds per mixture component):
            # at N = 40 550, d = 12, K = 878 from 32 components, 450 of 3000
            # sampled points have two centres within the bound in exact
            # arithmetic and 27 within 2^-19 |x| max|c|, and 20 labels differ
            # -- so the curated tests' 0.5 % cap on the count gives way here
            # to a check against gross breakage
            events.append(int(diff.sum()))
            assert diff.sum() <= max(2, 0.05 * rows.size), (N, d, K)
    record_property("label_events_per_float_case", events)
