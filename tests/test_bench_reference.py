"""The benchmark's reference arm (the oracle on the host cores) runs without
a GPU and prints one well-formed JSON line for every kind of workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,metric_word", [
    ("gmm-N1e4-d2-K16", "k-means++"),
    ("batch-512", "k-means++"),
    ("lloyd-gmm-N1e6-d32-K256", "Lloyd"),
    ("kmpar-gmm-N1e4-d2-K16", "k-means||"),
])
def test_reference_arm_prints_one_json_line(workload, metric_word):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", workload, "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, check=True, cwd=ROOT, timeout=600)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and metric_word in d["metric"]
    assert d["value"] > 0 and d["unit"] == "N*K*d/s" and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0
