"""Full-size workloads on the GPU, checked bit for bit on sampled entries the
oracle recomputes one by one, and by decryption of every output against the
plaintext predicate (a property that holds at any size).

The interval-validation query of the benchmark (D = 1,024, 134,144
bootstraps) runs by default.  The larger identifier-matching (D = 65,536,
4.1 M bootstraps) and 64-query coordinate-validation (~7.7 M bootstraps)
workloads take minutes and run when VELOPIR_FULL_SIZE=1."""
import os

import numpy as np
import pytest

import oracle
from gpu_common import encrypt_value_bits, gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu
FULL = os.environ.get("VELOPIR_FULL_SIZE") == "1"


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


@pytest.mark.skipif(not FULL, reason="full-size run: set VELOPIR_FULL_SIZE=1")
def test_idm32_d65536_full_size(paper_keys):
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    D = 65536
    w = synth.idm_workload(D, 32, distinct=True, payload=True)
    x = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["query"]], 32)[0], synth.lwe_material(32, substream=5))
    ids = w["ids"].astype(np.uint32)
    pay = w["payload"].astype(np.uint32)
    match = np.zeros((D, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 32, ids, D, None, 0, match)
    bits = vp.velopir_client_decrypt_bits(s, match)
    assert int(bits.sum()) == 1 and bits[w["planted"]] == 1
    sample = sorted({0, 12345, D - 1, w["planted"]} | set(range(7, D, 4099)))
    assert np.array_equal(match[sample], oracle.idm_batch(paper_keys, x, ids[sample]))
    agg = np.zeros((32, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 32, ids, D, pay, 32, agg)
    got = vp.velopir_client_decrypt_bits(s, agg)
    assert sum(int(b) << j for j, b in enumerate(got)) == int(pay[w["planted"]])


@pytest.mark.skipif(not FULL, reason="full-size run: set VELOPIR_FULL_SIZE=1")
def test_cov_64_queries_uneven_full_size(paper_keys):
    """64 coordinate queries, D log-uniform in [256, 16384], one merged program
    captured in a CUDA graph, autotuned tile shapes."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    vp.velopir_autotune(ctx.h)
    sizes = synth.log_uniform_sizes(64, 256, 16384, substream=9)
    qs, recs = [], []
    for q, D in enumerate(sizes):
        w = synth.cov_workload(int(D), substream=100 + q)
        cell = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["cell"]], 32)[0],
                                              synth.lwe_material(32, substream=200 + q))
        cells = w["cells"].astype(np.uint32)
        out = np.zeros((int(D), 631), dtype=np.uint32)
        qs.append((w, cell, cells, out))
        recs.append(vp.make_query(vp.VP_QUERY_COV, cell, cells, int(D), out))
    vp.velopir_query_batch(ctx.h, recs, use_graph=True)
    for q, (w, cell, cells, out) in enumerate(qs):
        bits = vp.velopir_client_decrypt_bits(s, out)
        assert np.array_equal(bits, (cells == w["cell"]).astype(np.uint32)), q
    for q in (0, 31, 63):
        w, cell, cells, out = qs[q]
        sample = sorted({0, len(cells) - 1, w["planted"]})
        assert np.array_equal(out[sample], oracle.cov_batch(paper_keys, cell, cells[sample]))
