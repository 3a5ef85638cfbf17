"""Parity checks of the CUDA seeding path against the FP64 oracle.

The oracle is replayed on the GPU's own trajectory (forced prefix = the GPU's
indices), so a single oracle run yields, for every draw, the oracle's own
choice and the FP64 prefix sums around the GPU's choice.  A draw passes if
the two agree, or if the GPU's choice lies within the tolerance band of the
prefix boundary between them (a "near-boundary event": every D^2 is within
``rtol`` relative, so every prefix sum is within ``rtol * T``; the band is
``band * T``).  D^2 must be within ``rtol`` relative elementwise, exact
where the oracle has 0, and phi within ``rtol`` relative.
"""
from __future__ import annotations

import numpy as np

import oracle

RTOL = 1e-5   # D^2 relative tolerance of the FP32 path
BAND = 2e-5   # draw band: two D^2 tolerances of T

# Near-tie bound of the tensor-core nearest-centre search (Lloyd assignment,
# k-means|| nearest candidate), which scores |c|^2 - 2 x.c with x and c split
# into two BF16 planes (x = xh + xl + rx, |xl| <= 2^-8 |x|, |rx| <= 2^-16 |x|,
# c alike) and x.c = xh.ch + xh.cl + xl.ch accumulated in FP32.  The dropped
# xl.cl, rx.c and x.rc are each at most 2^-16 |x||c| (Cauchy-Schwarz), FP32
# accumulation over 3 d / 16 MMA steps adds about d / 16 * 2^-23 |x||c|
# (2^-19 at d = 128): a score is within ~2^-14.4 |x||c| of exact, and the
# chosen centre's squared distance exceeds the nearest one's only when the
# two are within twice that.  The tests allow 2^-15 |x| max|c| -- below that
# worst case, at the scale the measured events reach (on GB300, at most
# 2^-17.8 over the test shapes) -- and at most 0.5 % of the points
# (measured: 0.03-0.16 %).
LABEL_BOUND = 2.0 ** -15
LABEL_EVENT_FRAC = 0.005


def check(points, K, seed, stream_id, gpu_idx, gpu_d2, gpu_phi=None, *, scales=None,
          dtype=None, exact=False, rtol=RTOL, band=BAND, status=None):
    """Compare one GPU seeding with the oracle; returns the near-boundary event count.

    ``exact``: integer-coordinate regime, where indices, D^2 and phi must be
    bit-identical (no events allowed).
    """
    gpu_idx = np.asarray(gpu_idx, dtype=np.int64)
    gpu_d2 = np.asarray(gpu_d2, dtype=np.float64)
    valid = gpu_idx[gpu_idx >= 0]
    r = oracle.seed(points, K, seed, stream_id, dtype=dtype, scales=scales,
                    forced=valid, draws=True)
    if status is not None:
        assert status == r["status"], (status, r["status"])
    if r["status"] == oracle.DEGENERATE:
        n = len(valid)
        assert np.all(gpu_idx[n:] == -1)
        assert np.all(r["idx"][n:] == -1)
    dr = r["draws"]
    assert gpu_idx[0] == dr["own"][0], (gpu_idx[0], dr["own"][0])
    events = 0
    for m in range(1, len(valid)):
        g, own = int(gpu_idx[m]), int(dr["own"][m])
        T, t = dr["T"][m], dr["t"][m]
        assert dr["P_at"][m] > dr["P_before"][m], f"draw {m}: index {g} has zero weight"
        if g == own:
            continue
        assert not exact, f"draw {m}: gpu {g} != oracle {own} in the exact regime"
        if g < own:
            ok = dr["P_at"][m] >= t - band * T
        else:
            ok = dr["P_before"][m] <= t + band * T
        assert ok, (f"draw {m}: gpu {g} oracle {own} t={t!r} T={T!r} "
                    f"P_before={dr['P_before'][m]!r} P_at={dr['P_at'][m]!r}")
        events += 1
    d2o = r["d2"]
    if exact:
        assert np.array_equal(gpu_d2, d2o), np.max(np.abs(gpu_d2 - d2o))
        if gpu_phi is not None:
            assert float(gpu_phi) == r["phi"], (float(gpu_phi), r["phi"])
    else:
        zero = d2o == 0
        assert np.all(gpu_d2[zero] == 0.0), "a zero D^2 of the oracle is nonzero on the GPU"
        err = np.abs(gpu_d2 - d2o)
        bad = err > rtol * d2o
        assert not bad.any(), (f"{bad.sum()} D^2 outside rtol; worst rel "
                               f"{np.max(err[~zero] / d2o[~zero]):.3e}")
        if gpu_phi is not None:
            assert abs(float(gpu_phi) - r["phi"]) <= rtol * r["phi"], (float(gpu_phi), r["phi"])
    return events
