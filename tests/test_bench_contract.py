"""The benchmark's reference arm (the oracle on the host cores) runs without a
GPU: its JSON line carries every key the benchmark contract names, and the
oracle's samples do not depend on its thread count."""
import json
import os
import subprocess
import sys

import numpy as np

import oracle
from paper_2103_02202_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "surface_d3", "--steps", "2", "--warmup", "1", "--cpu-shots", "8"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "shot-gates/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_oracle_samples_do_not_depend_on_threads():
    text = W.surface_code_memory(5, 3, 0.02)
    c = oracle.Circuit(text)
    shots = np.arange(300) * 7 + 11
    m1, d1 = c.sample(shots, 5, shot_offset=128, threads=1)
    m8, d8 = c.sample(shots, 5, shot_offset=128, threads=8)
    np.testing.assert_array_equal(m1, m8)
    np.testing.assert_array_equal(d1, d8)
