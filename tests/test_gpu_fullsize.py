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

import oracle
from gpu_common import encrypt_value_bits, gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def test_intv_d1024_full_size(paper_keys):
    """The benchmark's workload and launch configuration (autotuned NTT path)."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    vp.velopir_autotune(ctx.h)
    D = 1024
    w = synth.intv_workload(D)
    cx = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["x"]], 32)[0], synth.lwe_material(32, substream=1))
    cy = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["y"]], 32)[0], synth.lwe_material(32, substream=2))
    rects = np.ascontiguousarray(w["rects"], dtype=np.uint32)
    out = np.zeros((D, 631), dtype=np.uint32)
    vp.velopir_interval_query(ctx.h, cx, cy, rects, D, out)
    r = rects.astype(np.int64)
    want = ((r[:, 0] <= w["x"]) & (w["x"] < r[:, 1]) & (r[:, 2] <= w["y"]) & (w["y"] < r[:, 3])).astype(np.uint32)
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, out), want)
    sample = sorted({0, 1, D // 2, D - 1} | set(np.flatnonzero(want)[:2].tolist()))
    got = oracle.intv_batch(paper_keys, cx, cy, rects[sample].astype(np.uint64))
    assert np.array_equal(out[sample], got)
