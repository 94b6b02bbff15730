"""Failure detection without a GPU fault: a device wait that runs out is
reported as VELOPIR_ERR_TIMEOUT and the context stays usable; host-side
failures (bad arguments, an HBM budget too small for a request) return
status codes instead of crashing."""
import time

import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(paper_keys):
    ctx, s = gpu_ctx()
    t0 = time.perf_counter()
    rc = vp.velopir_selftest_wait_timeout(ctx.h)
    dt = time.perf_counter() - t0
    assert rc == -5, vp.velopir_last_error(ctx.h)        # VELOPIR_ERR_TIMEOUT
    assert 1.5 < dt < 30
    bits = synth.Stream(4, 2, 3).bits(4)
    inp = vp.velopir_client_encrypt_bits(s, bits, synth.lwe_material(4, seed=4)).reshape(2, 2, 631)
    out = np.zeros((2, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_AND, inp, out, 2)          # the context still works
    assert np.array_equal(out, oracle.gate_batch(paper_keys, oracle.AND, inp))


def test_budget_too_small_is_an_oom_status():
    km = synth.key_material()
    bk, ksk = vp.velopir_client_keygen(km)
    ctx = vp.Context(0, hbm_budget_bytes=64 << 20)     # smaller than the cloud key
    with pytest.raises(vp.VelopirError) as e:
        vp.velopir_load_cloud_key(ctx.h, bk, ksk)
    assert e.value.code == -3                           # VELOPIR_ERR_OOM
    ctx.close()


def test_query_without_key_is_a_nokey_status():
    ctx = vp.Context(0)
    x = np.zeros((8, 631), dtype=np.uint32)
    with pytest.raises(vp.VelopirError) as e:
        vp.velopir_id_match(ctx.h, x, 8, np.zeros(4, dtype=np.uint32), 4, None, 0, np.zeros((4, 631), np.uint32))
    assert e.value.code == -2
    with pytest.raises(vp.VelopirError):
        vp.velopir_id_match(ctx.h, x, 40, np.zeros(4, dtype=np.uint32), 4, None, 0, np.zeros((4, 631), np.uint32))
    ctx.close()
