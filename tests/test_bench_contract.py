"""The reference arm of bench.py (the oracle on the host cores) prints one
JSON line with the benchmark contract's keys and the same metric, unit and
config as the GPU arm; it needs no GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def reference_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-budget", "1"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT, env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_line_keys(reference_line):
    d = reference_line
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert cb["config1_full_circuit"]["decrypt_ok"] is True


def test_reference_and_gpu_arms_share_metric_unit_and_config(reference_line):
    sys.path.insert(0, ROOT)
    import bench
    assert reference_line["metric"] == bench.METRIC and reference_line["unit"] == bench.UNIT
    assert reference_line["config"] == bench.bench_config(1)
    assert reference_line["config"]["workload"] and "l2" in reference_line["config"]
