"""Seeded synthetic inputs for k-means++ seeding.

This module only draws data; it holds none of the seeding arithmetic, so the
CUDA path, the tests and the CPU oracle can all take their inputs from it.

The paper measures on unnamed two-dimensional data of 1-10 million points
(Section III) and publishes no dataset, so every workload here is a seeded
Gaussian mixture:

* ``gmm(...)``: ``n_comp`` components; means uniform in ``[-mean_box,
  mean_box]^d``; per-component isotropic sigma, fixed or uniform in
  ``sigma_range``; weights equal or Dirichlet(1); every point draws its
  component label i.i.d. (so point order is random).  numpy PCG64 generator,
  machine independent.  A fraction of the rows can be replaced by
  heavy-tailed 10 * Student-t(3) rows, centred at the origin or at their
  component's mean.
* ``gmm_torch(...)``: the same recipe drawn in chunks with a torch generator
  on a device, for the 10^7-10^8-point workloads that numpy draws too slowly.
* ``WORKLOADS``: the named workloads, with their sizes.
* ``batch_table(...)``: the 512-problem batch (N log-uniform in [1e3, 2e5], d
  from {8, 16, 32, 64, 128}, K log-uniform in [8, 256] clamped to N), drawn
  from ``numpy.random.default_rng(1000)``; problem p uses data seed p.
* ``integer_points(...)``: integer coordinates, for the regime where every
  D^2 and every prefix sum is exact in both FP32 and FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    d: int
    K: int
    n_comp: int
    mean_box: float
    sigma: tuple  # (lo, hi); lo == hi means fixed
    weights: str  # "equal" | "dirichlet"
    data_seed: int = 0
    draw_seed: int = 1
    outlier_frac: float = 0.0  # fraction replaced by 10 * Student-t(3) rows
    outlier_center: str = "zero"  # "zero" | "component": where those rows are centred


WORKLOADS = {
    # 16-component isotropic mixture, sigma 1, equal weights.
    "gmm-N1e4-d2-K16": Workload("gmm-N1e4-d2-K16", 10_000, 2, 16, 16, 10.0,
                                (1.0, 1.0), "equal"),
    # 256 components, means in [-50,50]^32, sigma U[0.5,2], Dirichlet(1) weights.
    "gmm-N1e6-d32-K256": Workload("gmm-N1e6-d32-K256", 1_000_000, 32, 256, 256,
                                  50.0, (0.5, 2.0), "dirichlet"),
    # Same recipe with 1024 components (precision form: FP32 vs BF16).
    "gmm-N1e7-d64-K1024": Workload("gmm-N1e7-d64-K1024", 10_000_000, 64, 1024,
                                   1024, 50.0, (0.5, 2.0), "dirichlet"),
    # 2048 components plus 10% heavy-tailed rows (FP32 vs BF16 vs FP8).
    "gmm-N2e7-d128-K2048-t3": Workload("gmm-N2e7-d128-K2048-t3", 20_000_000, 128,
                                       2048, 2048, 50.0, (0.5, 2.0), "dirichlet",
                                       outlier_frac=0.10),
    # The other reading of the heavy-tailed rows: each centred at the mean of
    # the component the row was drawn from, instead of at the origin.
    "gmm-N2e7-d128-K2048-t3c": Workload("gmm-N2e7-d128-K2048-t3c", 20_000_000, 128,
                                        2048, 2048, 50.0, (0.5, 2.0), "dirichlet",
                                        outlier_frac=0.10, outlier_center="component"),
}


def _mixture_params(rng: np.random.Generator, d: int, n_comp: int, mean_box: float,
                    sigma: tuple, weights: str):
    means = rng.uniform(-mean_box, mean_box, size=(n_comp, d))
    lo, hi = sigma
    sig = np.full(n_comp, lo) if lo == hi else rng.uniform(lo, hi, size=n_comp)
    if weights == "equal":
        w = np.full(n_comp, 1.0 / n_comp)
    else:
        w = rng.dirichlet(np.ones(n_comp))
    return means, sig, w


def gmm(N: int, d: int, n_comp: int, seed: int, mean_box: float = 50.0,
        sigma: tuple = (0.5, 2.0), weights: str = "dirichlet",
        outlier_frac: float = 0.0, outlier_center: str = "zero") -> np.ndarray:
    """Gaussian-mixture points, float32 [N, d] (numpy PCG64, seeded).

    ``outlier_frac`` of the rows, chosen without replacement, are replaced by
    10 * Student-t(3) draws, centred at the origin (``outlier_center`` "zero")
    or at the mean of the row's component ("component").
    """
    rng = np.random.default_rng(seed)
    means, sig, w = _mixture_params(rng, d, n_comp, mean_box, sigma, weights)
    labels = rng.choice(n_comp, size=N, p=w)
    x = np.empty((N, d), dtype=np.float32)
    chunk = max(1, (1 << 22) // max(d, 1))
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        lab = labels[s:e]
        z = rng.standard_normal((e - s, d))
        x[s:e] = (means[lab] + sig[lab, None] * z).astype(np.float32)
    if outlier_frac > 0.0:
        n_out = int(round(outlier_frac * N))
        rows = rng.choice(N, size=n_out, replace=False)
        t = 10.0 * rng.standard_t(3.0, size=(n_out, d))
        if outlier_center == "component":
            t = t + means[labels[rows]]
        elif outlier_center != "zero":
            raise ValueError(f"unknown outlier centre {outlier_center!r}")
        x[rows] = t.astype(np.float32)
    return x


def gmm_torch(N: int, d: int, n_comp: int, seed: int, device, mean_box: float = 50.0,
              sigma: tuple = (0.5, 2.0), weights: str = "dirichlet",
              outlier_frac: float = 0.0, outlier_center: str = "zero"):
    """The ``gmm`` recipe drawn with a torch generator on ``device`` (float32 [N, d]).

    Mixture parameters come from numpy (seeded); the per-point labels, normals
    and outliers from ``torch.Generator(device).manual_seed(seed)``.
    """
    import torch

    rng = np.random.default_rng(seed)
    means, sig, w = _mixture_params(rng, d, n_comp, mean_box, sigma, weights)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    means_t = torch.as_tensor(means, dtype=torch.float32, device=device)
    sig_t = torch.as_tensor(sig, dtype=torch.float32, device=device)
    w_t = torch.as_tensor(w, dtype=torch.float64, device=device)
    if outlier_center not in ("zero", "component"):
        raise ValueError(f"unknown outlier centre {outlier_center!r}")
    x = torch.empty((N, d), dtype=torch.float32, device=device)
    keep_labels = outlier_frac > 0.0 and outlier_center == "component"
    labels = torch.empty(N, dtype=torch.int64, device=device) if keep_labels else None
    chunk = max(1, (1 << 26) // d)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        lab = torch.multinomial(w_t, e - s, replacement=True, generator=g)
        z = torch.randn((e - s, d), generator=g, device=device, dtype=torch.float32)
        x[s:e] = means_t[lab] + sig_t[lab, None] * z
        if keep_labels:
            labels[s:e] = lab
    if outlier_frac > 0.0:
        n_out = int(round(outlier_frac * N))
        rows = torch.randperm(N, generator=g, device=device)[:n_out]
        # Student-t(3) = Z / sqrt(chi2_3 / 3), chi2_3 = sum of 3 squared normals.
        for s in range(0, n_out, chunk):
            e = min(n_out, s + chunk)
            z = torch.randn((e - s, d), generator=g, device=device)
            c = torch.randn((e - s, d, 3), generator=g, device=device).square().sum(-1)
            t = 10.0 * z / torch.sqrt(c / 3.0)
            if keep_labels:
                t = t + means_t[labels[rows[s:e]]]
            x[rows[s:e]] = t
    return x


def workload_points(wl: Workload, device=None):
    """Points of a named workload: numpy (device None) or a torch tensor."""
    if device is None:
        return gmm(wl.N, wl.d, wl.n_comp, wl.data_seed, wl.mean_box, wl.sigma,
                   wl.weights, wl.outlier_frac, wl.outlier_center)
    return gmm_torch(wl.N, wl.d, wl.n_comp, wl.data_seed, device, wl.mean_box,
                     wl.sigma, wl.weights, wl.outlier_frac, wl.outlier_center)


@dataclass(frozen=True)
class Problem:
    p: int
    N: int
    d: int
    K: int


def batch_table(n_problems: int = 512, meta_seed: int = 1000,
                n_range=(1_000, 200_000), dims=(8, 16, 32, 64, 128),
                k_range=(8, 256)) -> list:
    """Sizes of the uneven batch: N and K log-uniform, d uniform over ``dims``."""
    rng = np.random.default_rng(meta_seed)
    out = []
    for p in range(n_problems):
        N = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        d = int(dims[rng.integers(len(dims))])
        K = int(round(math.exp(rng.uniform(math.log(k_range[0]), math.log(k_range[1])))))
        out.append(Problem(p, N, d, min(K, N)))
    return out


def batch_problem_points(pr: Problem) -> np.ndarray:
    """Points of batch problem ``pr``: a K-component mixture, data seed p."""
    return gmm(pr.N, pr.d, pr.K, pr.p, 50.0, (0.5, 2.0), "dirichlet")


def integer_points(N: int, d: int, seed: int, lo: int = -64, hi: int = 64,
                   n_comp: int = 0) -> np.ndarray:
    """Integer coordinates in [lo, hi] stored as float32 [N, d].

    With |x| <= 64 and d <= 128 every squared distance is below 2^21, exact in
    FP32 (and in BF16 storage, since integers up to 256 are exact there), and
    every FP64 prefix sum over up to 2^31 points is exact.  ``n_comp`` > 0
    clusters the integers around that many integer centres.
    """
    rng = np.random.default_rng(seed)
    if n_comp <= 0:
        return rng.integers(lo, hi + 1, size=(N, d)).astype(np.float32)
    span = (hi - lo) // 4
    centres = rng.integers(lo + span, hi - span + 1, size=(n_comp, d))
    lab = rng.integers(n_comp, size=N)
    x = centres[lab] + rng.integers(-span, span + 1, size=(N, d))
    return np.clip(x, lo, hi).astype(np.float32)
