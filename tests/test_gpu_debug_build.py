"""The KPP_DEBUG build of the library (index checks before every hot-path
memory access of the seeding kernels, and a check that each tensor-core
assignment launch's shared-memory plan fits it; a failed check reported as
the device status KPP_ERR_BOUNDS instead of a memory fault -- the stand-in
for a sanitizer, which this GPU does not run): the exact-regime parity cases
of every seeding form, of the Lloyd iteration (both assignment kernels) and
of k-means|| run under it, in a child process that loads the debug library,
and must pass -- every call's status is read, so one index out of bounds
anywhere fails them."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    "tests/test_gpu_parity.py::test_exact_regime_bit_identical",
    "tests/test_gpu_parity.py::test_persistent_options_exact",
    "tests/test_gpu_parity.py::test_every_lanes_per_row_variant",
    "tests/test_gpu_parity.py::test_degenerate_data_reports_status",
    "tests/test_gpu_parity.py::test_k1_and_k_equals_n",
    "tests/test_gpu_parity.py::test_float_regime_low_precision_storage",
    "tests/test_gpu_small.py",
    "tests/test_gpu_shard.py::test_sharded_integer_regime_bit_identical",
    "tests/test_gpu_shard.py::test_uneven_shards_and_a_one_row_shard",
    "tests/test_gpu_batched.py",
    "tests/test_gpu_exact_draws.py::test_exact_decisions_integer_regime",
    "tests/test_gpu_recompute.py",
    "tests/test_gpu_lloyd.py::test_integer_regime_bit_identical",
    "tests/test_gpu_lloyd.py::test_pair_form_integer_regime_bit_identical",
    "tests/test_gpu_lloyd.py::test_exact_ties_take_the_smallest_centre_index",
    "tests/test_gpu_kmpar.py::test_integer_regime_matches_oracle_exactly",
]


def _env():
    env = dict(os.environ)
    env["KPP_DEBUG"] = "1"
    return env


def test_debug_library_is_the_one_loaded():
    out = subprocess.run(
        [sys.executable, "-c",
         "import paper_1908_02136_gb300 as k; k.load_library(); print(k.library_path())"],
        capture_output=True, text=True, check=True, cwd=ROOT, env=_env(), timeout=900)
    assert out.stdout.strip().endswith(os.path.join("_build_debug", "libkpp.so"))


def test_parity_under_the_debug_build():
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", *CASES],
                       capture_output=True, text=True, cwd=ROOT, env=_env(), timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
