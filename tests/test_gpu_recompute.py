"""The paper's own seeding step as a comparison form (KPP_FORM_RECOMPUTE):
every pass recomputes each point's distance to all seeds chosen so far
(Section II) instead of to the newest one.  The minimum of the same FP32
distances is the same number, so indices, D^2 and phi must be bit-identical
to the streamed form's, and to the oracle's in the exact-arithmetic regime."""
import numpy as np
import pytest
import torch

import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.mark.parametrize("N,d,K,dtype", [(20_000, 32, 24, "f32"), (9_001, 2, 16, "f32"),
                                         (12_345, 64, 20, "bf16"), (5_000, 7, 12, "f32"),
                                         (8_000, 128, 10, "fp8")])
def test_recompute_equals_incremental(N, d, K, dtype):
    x = torch.from_numpy(datagen.gmm(N, d, K, seed=N)).to(DEV)
    scales = None
    if dtype == "bf16":
        x = kpp.quantize(x, "bf16")
    elif dtype == "fp8":
        x, scales = kpp.quantize(x, "fp8")
    a = kpp.seed(x, K, 3, 1, dtype=dtype, row_scales=scales, opts={"form": kpp.FORM_STREAMED})
    b = kpp.seed(x, K, 3, 1, dtype=dtype, row_scales=scales, opts={"form": kpp.FORM_RECOMPUTE})
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_recompute_integer_regime_matches_oracle():
    x = datagen.integer_points(15_000, 16, seed=4, n_comp=8)
    idx, d2, phi = kpp.seed(torch.from_numpy(x).to(DEV), 32, 9, 2,
                            opts={"form": kpp.FORM_RECOMPUTE})
    parity.check(x, 32, 9, 2, idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0]),
                 exact=True)


def test_recompute_is_reported_by_describe():
    with torch.cuda.device(DEV):
        st, plan = kpp.kpp_describe(10_000, 32, 16, kpp.F32, {"form": kpp.FORM_RECOMPUTE})
    assert st == kpp.OK and plan.form == kpp.FORM_RECOMPUTE and plan.launches == 16
