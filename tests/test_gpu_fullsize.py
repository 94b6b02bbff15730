"""The benchmark's workload at full size on the GPU (interval validation,
D = 1,024, 134,144 bootstraps, the autotuned NTT path), checked bit for bit
on sampled entries the oracle recomputes one by one, and by decryption of
every output against the plaintext predicate (a property that holds at any
size).  The identifier-matching and multi-query coordinate shapes run in
tests/test_gpu_scale.py at sizes that reach every full-size code path, with
traced gates recomputed by the oracle; config_bench runs them at full size
and decrypts every output."""
import numpy as np
import pytest

from gpu_common import fullsize_inputs, fullsize_oracle, gpu_ctx
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def test_intv_d1024_full_size(paper_keys):
    """The benchmark's workload and launch configuration (autotuned NTT path)."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    vp.velopir_autotune(ctx.h)
    f = fullsize_inputs(s)
    out = np.zeros((f["D"], 631), dtype=np.uint32)
    vp.velopir_interval_query(ctx.h, f["cx"], f["cy"], f["rects"], f["D"], out)
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, out), f["want"])
    assert f["want"].sum() >= 1
    assert np.array_equal(out[f["sample"]], fullsize_oracle(paper_keys))
