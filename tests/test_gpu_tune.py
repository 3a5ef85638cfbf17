"""GPU tests of the autotuner (kpp_tune, through the C ABI): the winner is a
valid plan, it is recorded for the automatic choice of the same shape and
forgotten on kpp_tune_clear, seeding with it still matches the FP64 oracle
exactly in the exact-arithmetic regime, and a degenerate input or a
workspace that holds no candidate is reported."""
import ctypes

import numpy as np
import pytest
import torch

import parity
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(autouse=True)
def clean_table():
    kpp.kpp_tune_clear()
    yield
    kpp.kpp_tune_clear()


def _plan(N, d, K, dt, opts=None):
    st, p = kpp.kpp_describe(N, d, K, dt, opts)
    assert st == kpp.OK
    return (p.form, p.grid, p.lanes_per_row, p.d2_in_smem, p.rows_per_cta, p.cached_rows_per_cta)


@pytest.mark.parametrize("N,d,K", [(20_011, 32, 24), (3_001, 8, 12), (150_007, 64, 16)])
def test_tuned_choice_is_recorded_and_seeds_exactly(N, d, K):
    x_np = datagen.integer_points(N, d, seed=N, n_comp=8)
    x = torch.from_numpy(x_np).to(DEV)
    with torch.cuda.device(DEV):
        before = _plan(N, d, K, kpp.F32)
    best, ms = kpp.tune(x, K, passes=8)
    assert best["form"] in (kpp.FORM_STREAMED, kpp.FORM_PERSISTENT, kpp.FORM_SMALL)
    assert ms > 0.0
    with torch.cuda.device(DEV):
        tuned = _plan(N, d, K, kpp.F32, best)
        auto = _plan(N, d, K, kpp.F32)
        assert auto == tuned  # the automatic choice is now the tuner's
        # other shapes keep the heuristic choice
        assert _plan(N + 1, d, K, kpp.F32) == _plan(N + 1, d, K, kpp.F32, {"form": 0})
    idx, d2, phi = kpp.seed(x, K, 5, 3)
    parity.check(x_np, K, 5, 3, idx.cpu().numpy(), d2.cpu().numpy(), float(phi.cpu()[0]),
                 exact=True)
    kpp.kpp_tune_clear()
    with torch.cuda.device(DEV):
        assert _plan(N, d, K, kpp.F32) == before


def test_explicit_options_are_not_overridden():
    N, d, K = 20_011, 32, 24
    x = torch.from_numpy(datagen.integer_points(N, d, seed=1)).to(DEV)
    kpp.tune(x, K, passes=4)
    with torch.cuda.device(DEV):
        st, p = kpp.kpp_describe(N, d, K, kpp.F32, {"form": kpp.FORM_STREAMED})
        assert st == kpp.OK and p.form == kpp.FORM_STREAMED


def test_bf16_tuning():
    N, d, K = 40_009, 64, 16
    x = torch.from_numpy(datagen.gmm(N, d, 16, seed=3)).to(DEV)
    q = kpp.quantize(x, "bf16")
    best, ms = kpp.tune(q, K, dtype="bf16", passes=4)
    assert ms > 0.0
    idx, d2, phi = kpp.seed(q, K, 1, dtype="bf16")
    assert len(set(idx.cpu().tolist())) == K


def test_degenerate_data_is_reported_and_not_recorded():
    x = torch.zeros((5_000, 16), device=DEV)
    with pytest.raises(kpp.KppError) as e:
        kpp.tune(x, 8, passes=4)
    assert e.value.status == kpp.ERR_DEGENERATE
    with torch.cuda.device(DEV):
        assert _plan(5_000, 16, 8, kpp.F32) == _plan(5_000, 16, 8, kpp.F32, {"form": 0})


def test_workspace_too_small_for_every_candidate():
    N, d, K = 20_011, 32, 8
    x = torch.from_numpy(datagen.integer_points(N, d, seed=2)).to(DEV)
    idx = torch.empty(K, dtype=torch.int64, device=DEV)
    d2 = torch.empty(N, dtype=torch.float32, device=DEV)
    ws = torch.empty(256, dtype=torch.uint8, device=DEV)
    best = kpp.Options()
    with torch.cuda.device(DEV):
        st = kpp.kpp_tune(x.data_ptr(), None, N, d, K, kpp.F32, idx.data_ptr(), d2.data_ptr(),
                          ws.data_ptr(), ws.numel(),
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), 4, best)
    assert st == kpp.ERR_UNSUPPORTED


_CACHE_CHILD = r"""
import os, sys, json, numpy as np, torch
sys.path.insert(0, os.getcwd())
import paper_1908_02136_gb300 as kpp
from paper_1908_02136_gb300 import datagen
N, d, K = 20_011, 32, 24
x = torch.from_numpy(datagen.integer_points(N, d, seed=N, n_comp=8)).to("cuda:0")
if sys.argv[1] == "tune":
    best, ms = kpp.tune(x, K, passes=8)
    print(json.dumps({"best": best}))
else:
    st, p = kpp.kpp_describe(N, d, K, kpp.F32)
    assert st == kpp.OK
    print(json.dumps({"plan": [p.form, p.grid, p.lanes_per_row, p.rows_per_cta,
                               p.cached_rows_per_cta]}))
"""


def test_tuning_cache_file_carries_the_winner_to_a_new_process(tmp_path):
    """KPP_TUNE_CACHE: one process tunes and appends its winner to the file;
    a second process, which does not tune, makes the same automatic choice."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, KPP_TUNE_CACHE=str(cache))

    def child(mode):
        r = subprocess.run([sys.executable, "-c", _CACHE_CHILD, mode], capture_output=True,
                           text=True, cwd=root, env=env, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        return json.loads(r.stdout.strip().splitlines()[-1])

    best = child("tune")["best"]
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("kpp-tune 1 ")
    plan = child("describe")["plan"]
    with torch.cuda.device(DEV):
        st, p = kpp.kpp_describe(20_011, 32, 24, kpp.F32, best)
    assert st == kpp.OK
    assert plan == [p.form, p.grid, p.lanes_per_row, p.rows_per_cta, p.cached_rows_per_cta]
