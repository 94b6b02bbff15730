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


def test_bench_query_schedule_on_the_host():
    """The benchmark's step (IntV, D = 1,024) as the scheduler issues it, by
    the host dry run: 134,144 blind rotations, the plaintext answer, and the
    wave-filled plan of 36 launches of two full 12-wide waves, one of one
    wave and a 992-gate tail -- 74 waves, where its 34 as-soon-as-possible
    layers would take 99."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_2506_12761_gb300 import synth
    from paper_2506_12761_gb300 import velopir as vp
    w = synth.intv_workload(bench.D)
    rects = np.ascontiguousarray(w["rects"], dtype=np.uint32)
    bits = lambda v: np.array([(int(v) >> i) & 1 for i in range(32)], dtype=np.uint32)
    wave = 152 * 12
    out, sizes = vp.velopir_plan_query(vp.VP_QUERY_INTV, rects, bench.D, bits(w["x"]), bits(w["y"]), wave=wave)
    r = rects.astype(np.int64)
    want = ((r[:, 0] <= w["x"]) & (w["x"] < r[:, 1]) & (r[:, 2] <= w["y"]) & (w["y"] < r[:, 3])).astype(np.uint32)
    assert np.array_equal(out, want)
    assert sum(sizes) == bench.BOOTSTRAPS_PER_STEP == 134144
    assert sorted(sizes) == [992, 1824] + [2 * wave] * 36
    _, layers = vp.velopir_plan_query(vp.VP_QUERY_INTV, rects, bench.D, bits(w["x"]), bits(w["y"]), wave=0)
    assert len(layers) == 34
    assert sum(-(-s // wave) for s in layers) == 99 and sum(-(-s // wave) for s in sizes) == 74
