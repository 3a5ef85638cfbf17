"""GPU parity of the batching form (kpp_seed_batched, through the C ABI):
every problem of a batch against the FP64 oracle, for problems run by teams
of CTAs and by single CTAs, every stored dtype, degenerate problems inside a
batch, and the 512-problem workload (oracle parity on a sample, invariants
on every problem)."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _store(x_np, dtype):
    x = torch.from_numpy(x_np).to(DEV)
    if dtype == "f32":
        return x, None, x_np
    if dtype == "bf16":
        q = kpp.quantize(x, "bf16")
        return q, None, q.cpu().numpy().view(np.uint16)
    q, s = kpp.quantize(x, "fp8")
    return q, s, q.cpu().numpy()


def _run(problems, dtype="f32", opts=None, check=True):
    """problems: list of (points np, K, seed, stream). Returns stored np, scales, results."""
    stored, scales, stored_np = zip(*[_store(x, dtype) for x, _, _, _ in problems])
    outs, ws = kpp.seed_batched(list(stored), [K for _, K, _, _ in problems],
                                [s for _, _, s, _ in problems],
                                [st for _, _, _, st in problems], dtype=dtype,
                                row_scales=None if scales[0] is None else list(scales),
                                opts=opts, check=check)
    torch.cuda.synchronize()
    res = [(i.cpu().numpy(), d.cpu().numpy(), float(p.cpu()[0])) for i, d, p in outs]
    sc = [None if s is None else s.cpu().numpy() for s in scales]
    return stored_np, sc, res


def _mixed(exact, seed=0):
    """A few large problems (teams) and many small ones (queue), d in the built set."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(6):
        N = int(rng.integers(60_000, 120_000))
        d = int(rng.choice([16, 32, 64]))
        K = int(rng.integers(20, 48))
        x = (datagen.integer_points(N, d, seed=100 + i, n_comp=8) if exact
             else datagen.gmm(N, d, K, seed=100 + i))
        probs.append((x, K, 1, i))
    for i in range(40):
        N = int(rng.integers(300, 6000))
        d = int(rng.choice([2, 4, 8, 16, 32, 64, 128]))
        K = int(rng.integers(1, min(64, N)))
        x = (datagen.integer_points(N, d, seed=200 + i, n_comp=6) if exact
             else datagen.gmm(N, d, max(K, 2), seed=200 + i))
        probs.append((x, K, 1, 6 + i))
    return probs


def test_batched_exact_regime_bit_identical():
    probs = _mixed(exact=True)
    st, sc, res = _run(probs, opts={"min_rows_per_cta": 1024})
    for (x, K, seed, stream), s_np, (idx, d2, phi) in zip(probs, st, res):
        parity.check(s_np, K, seed, stream, idx, d2, phi, exact=True)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_batched_float_regime(dtype):
    probs = _mixed(exact=False, seed=1)
    st, sc, res = _run(probs, dtype=dtype, opts={"min_rows_per_cta": 1024})
    events = 0
    for (x, K, seed, stream), s_np, scl, (idx, d2, phi) in zip(probs, st, sc, res):
        events += parity.check(s_np, K, seed, stream, idx, d2, phi, scales=scl)
    assert events <= 3


def test_batched_matches_single_problem_calls_in_exact_regime():
    probs = _mixed(exact=True, seed=2)[:20]
    st, sc, res = _run(probs, opts={"min_rows_per_cta": 2048})
    for (x, K, seed, stream), (idx, d2, phi) in zip(probs, res):
        i1, d1, p1 = kpp.seed(torch.from_numpy(x).to(DEV), K, seed, stream)
        assert np.array_equal(idx, i1.cpu().numpy())
        assert np.array_equal(d2, d1.cpu().numpy())
        assert phi == float(p1.cpu()[0])


def test_degenerate_problem_does_not_stop_the_batch():
    base = np.array([[0, 0, 0, 0], [1, 2, 3, 4], [5, 5, 5, 5]], np.float32)
    bad = np.repeat(base, [300, 300, 300], axis=0)
    probs = [(datagen.gmm(5000, 8, 8, seed=1), 10, 1, 0), (bad, 6, 1, 1),
             (datagen.gmm(90_000, 32, 16, seed=2), 24, 1, 2)]
    with pytest.raises(kpp.KppError) as e:
        _run(probs)
    assert e.value.status == kpp.ERR_DEGENERATE
    st, sc, res = _run(probs, check=False)
    assert np.all(res[1][0][3:] == -1) and res[1][2] == 0.0
    for k in (0, 2):
        x, K, seed, stream = probs[k]
        parity.check(st[k], K, seed, stream, *res[k])
    parity.check(st[1], 6, 1, 1, *res[1], exact=True, status=oracle.DEGENERATE)


def test_unsupported_dimension_is_rejected():
    x = torch.zeros((100, 3), device=DEV)
    with pytest.raises(kpp.KppError) as e:
        kpp.seed_batched([x], [4], [1])
    assert e.value.status == kpp.ERR_UNSUPPORTED  # no batched specialisation for d = 3


@pytest.mark.slow
def test_batch_workload_512_problems():
    table = datagen.batch_table()
    xs = [datagen.batch_problem_points(pr) for pr in table]
    probs = [(x, pr.K, 1, pr.p) for x, pr in zip(xs, table)]
    st, sc, res = _run(probs)
    rng = np.random.default_rng(7)
    sample = set(rng.choice(len(probs), 24, replace=False).tolist())
    events = 0
    for k, ((x, K, seed, stream), (idx, d2, phi)) in enumerate(zip(probs, res)):
        assert np.all((idx >= 0) & (idx < len(x))) and len(set(idx.tolist())) == K
        assert np.all(d2[idx] == 0.0) and np.all(d2 >= 0)
        assert abs(phi - d2.astype(np.float64).sum()) <= 1e-5 * phi
        if k in sample:
            events += parity.check(x, K, seed, stream, idx, d2, phi)
    assert events <= 2
