"""The synthetic input recipe (no GPU): seeded determinism, the named
workloads' sizes, the mixture's structure (components inside the mean box,
the per-component spread, mixture weights), the heavy-tailed rows, the batch
table's ranges and the exact-arithmetic integer points.  The torch-generated
form of the recipe is checked on the CPU device."""
import numpy as np
import pytest

from paper_1908_02136_gb300 import datagen


def test_named_workloads():
    w = datagen.WORKLOADS
    assert (w["gmm-N1e4-d2-K16"].N, w["gmm-N1e4-d2-K16"].d, w["gmm-N1e4-d2-K16"].K) == (10_000, 2, 16)
    assert (w["gmm-N1e6-d32-K256"].N, w["gmm-N1e6-d32-K256"].d) == (1_000_000, 32)
    assert w["gmm-N1e7-d64-K1024"].K == 1024 and w["gmm-N1e7-d64-K1024"].n_comp == 1024
    big = w["gmm-N2e7-d128-K2048-t3"]
    assert (big.N, big.d, big.K, big.outlier_frac) == (20_000_000, 128, 2048, 0.10)
    alt = datagen.WORKLOADS["gmm-N2e7-d128-K2048-t3c"]
    assert (alt.N, alt.d, alt.K, alt.outlier_center) == (20_000_000, 128, 2048, "component")
    for name, wl in w.items():
        assert wl.name == name and wl.K <= wl.N and wl.draw_seed == 1


def test_gmm_is_seeded_and_shaped():
    a = datagen.gmm(5000, 8, 4, seed=3)
    b = datagen.gmm(5000, 8, 4, seed=3)
    c = datagen.gmm(5000, 8, 4, seed=4)
    assert a.dtype == np.float32 and a.shape == (5000, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_gmm_components_lie_in_the_box_with_their_spread():
    # one well-separated component per corner region: recover the means and
    # spreads from the points nearest each true mean
    rng = np.random.default_rng(5)
    means, sig, w = datagen._mixture_params(rng, 3, 6, 50.0, (0.5, 2.0), "dirichlet")
    assert np.all(np.abs(means) <= 50.0)
    assert np.all((sig >= 0.5) & (sig <= 2.0))
    assert w.sum() == pytest.approx(1.0) and np.all(w > 0)
    x = datagen.gmm(60_000, 3, 6, seed=5)
    d2 = ((x[:, None, :].astype(np.float64) - means[None]) ** 2).sum(-1)
    lab = d2.argmin(1)
    counts = np.bincount(lab, minlength=6) / x.shape[0]
    np.testing.assert_allclose(counts, w, atol=0.02)
    for k in range(6):
        if counts[k] > 0.05:
            pts = x[lab == k].astype(np.float64)
            np.testing.assert_allclose(pts.mean(0), means[k], atol=0.2)
            assert pts.std(0).mean() == pytest.approx(sig[k], rel=0.1)


def test_equal_weights_and_fixed_sigma():
    rng = np.random.default_rng(0)
    means, sig, w = datagen._mixture_params(rng, 2, 16, 10.0, (1.0, 1.0), "equal")
    assert np.all(sig == 1.0) and np.allclose(w, 1 / 16)
    assert np.all(np.abs(means) <= 10.0)


def test_heavy_tailed_rows():
    x = datagen.gmm(20_000, 4, 3, seed=1, outlier_frac=0.10)
    y = datagen.gmm(20_000, 4, 3, seed=1, outlier_frac=0.0)
    # the mixture part is drawn first, so exactly the replaced rows differ
    changed = np.any(x != y, axis=1)
    assert changed.sum() == 2000
    # Student-t(3) x 10: heavy tails well beyond the mixture's box
    assert np.abs(x[changed]).max() > 100.0 and np.abs(y).max() < 60.0


def test_batch_table_ranges():
    t = datagen.batch_table()
    assert len(t) == 512 and [p.p for p in t] == list(range(512))
    assert all(1_000 <= p.N <= 200_000 for p in t)
    assert {p.d for p in t} == {8, 16, 32, 64, 128}
    assert all(8 <= p.K <= 256 and p.K <= p.N for p in t)
    assert t == datagen.batch_table()
    x = datagen.batch_problem_points(t[7])
    assert x.shape == (t[7].N, t[7].d) and x.dtype == np.float32


def test_integer_points():
    x = datagen.integer_points(1000, 5, seed=2)
    assert x.dtype == np.float32 and np.all(x == np.round(x))
    assert x.min() >= -64 and x.max() <= 64
    y = datagen.integer_points(1000, 5, seed=2, n_comp=4)
    assert np.all(y == np.round(y)) and y.min() >= -64 and y.max() <= 64


def test_torch_form_of_the_recipe_on_cpu():
    torch = pytest.importorskip("torch")
    a = datagen.gmm_torch(20_000, 4, 3, 7, "cpu")
    b = datagen.gmm_torch(20_000, 4, 3, 7, "cpu")
    assert a.dtype == torch.float32 and tuple(a.shape) == (20_000, 4)
    assert torch.equal(a, b)
    # same mixture parameters as the numpy form: the component means
    rng = np.random.default_rng(7)
    means, sig, w = datagen._mixture_params(rng, 4, 3, 50.0, (0.5, 2.0), "dirichlet")
    x = a.numpy().astype(np.float64)
    lab = ((x[:, None, :] - means[None]) ** 2).sum(-1).argmin(1)
    for k in range(3):
        if (lab == k).mean() > 0.05:
            np.testing.assert_allclose(x[lab == k].mean(0), means[k], atol=0.2)
    o = datagen.gmm_torch(20_000, 4, 3, 7, "cpu", outlier_frac=0.1)
    assert (o != a).any(dim=1).sum().item() == 2000


def test_heavy_tailed_rows_centred_at_their_component():
    x = datagen.gmm(20_000, 4, 3, seed=1, outlier_frac=0.10, outlier_center="component")
    y = datagen.gmm(20_000, 4, 3, seed=1, outlier_frac=0.10)
    z = datagen.gmm(20_000, 4, 3, seed=1)
    changed = np.any(x != z, axis=1)
    assert changed.sum() == 2000 and np.array_equal(changed, np.any(y != z, axis=1))
    # the same t draws, shifted by the row's component mean: the shift is one
    # of the three means for every replaced row
    rng = np.random.default_rng(1)
    means, _, _ = datagen._mixture_params(rng, 4, 3, 50.0, (0.5, 2.0), "dirichlet")
    shift = (x[changed].astype(np.float64) - y[changed].astype(np.float64))
    dist = np.abs(shift[:, None, :] - means[None]).max(-1).min(1)
    assert np.all(dist < 1e-3)
    with pytest.raises(ValueError):
        datagen.gmm(100, 2, 2, seed=0, outlier_frac=0.1, outlier_center="nowhere")


def test_torch_form_centres_outliers_at_their_component():
    torch = pytest.importorskip("torch")
    a = datagen.gmm_torch(20_000, 4, 3, 7, "cpu", outlier_frac=0.1)
    b = datagen.gmm_torch(20_000, 4, 3, 7, "cpu", outlier_frac=0.1, outlier_center="component")
    rng = np.random.default_rng(7)
    means, _, _ = datagen._mixture_params(rng, 4, 3, 50.0, (0.5, 2.0), "dirichlet")
    changed = (a != b).any(dim=1).numpy()
    assert 1_500 < changed.sum() <= 2_000  # rows whose shift is 0 in float32 stay equal
    shift = (b.numpy()[changed] - a.numpy()[changed]).astype(np.float64)
    assert np.all(np.abs(shift[:, None, :] - means[None]).max(-1).min(1) < 1e-3)
