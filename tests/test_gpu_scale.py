"""Identifier matching with payload aggregation and many uneven coordinate
queries under one captured graph, at sizes that reach every full-size code
path in a few minutes, checked three ways:

  * per gate: the gate trace records >= 4,096 gates sampled in every launch
    (so every level of the aggregation tree is reached), and the oracle
    recomputes each one from its recorded inputs and pre-combination;
  * per entry: whole entries recomputed by the oracle from the query's own
    ciphertexts (no GPU intermediate involved);
  * per output: every output decrypts to its plaintext answer."""
import numpy as np
import pytest

import oracle
from gpu_common import check_trace, gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu
TRACE_SEED = 20250615


def fanin_nodes(D, g):
    nodes, k = 0, 1
    while k < D:
        nodes += sum(1 for i in range(0, D, g * k) if sum(1 for q in range(g) if i + q * k < D) >= 2)
        k *= g
    return nodes


def idm_inputs(s, D):
    w = synth.idm_workload(D, 32, distinct=True, payload=True, substream=21)
    x = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["query"]], 32)[0], synth.lwe_material(32, substream=22))
    return w, x, w["ids"].astype(np.uint32), w["payload"].astype(np.uint32)


def test_idm32_d8192_match_bits_and_pairwise_aggregation_traced(paper_keys):
    """Config 3's circuit (31-AND trees, payload zero-out, Section 5's pairwise
    HomSum: 13 XOR levels) at D = 8,192: 516,064 bootstraps."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    vp.velopir_autotune(ctx.h)
    D = 8192
    w, x, ids, pay = idm_inputs(s, D)
    match = np.zeros((D, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 32, ids, D, None, 0, match)
    bits = vp.velopir_client_decrypt_bits(s, match)
    assert int(bits.sum()) == 1 and bits[w["planted"]] == 1
    sample = sorted({0, 1, 4097, D - 1, w["planted"]})
    assert np.array_equal(match[sample], oracle.idm_batch(paper_keys, x, ids[sample]))

    vp.velopir_trace_start(ctx.h, TRACE_SEED, 32, 125, 8192)      # >= 516,064 / 125 = 4,129 gates
    agg = np.zeros((32, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 32, ids, D, pay, 32, agg)
    recs = vp.velopir_trace_stop(ctx.h, 8192)
    assert len(recs) < 8192, "the trace buffer filled up: later launches were not sampled"
    got = vp.velopir_client_decrypt_bits(s, agg)
    assert sum(int(b) << j for j, b in enumerate(got)) == int(pay[w["planted"]])
    check_trace(paper_keys, recs, 4096)
    # the last gates of the tree (the outputs) are among the traced ones
    outs = {bytes(o) for o in agg}
    assert sum(bytes(r) in outs for r in recs["out"]) >= 1


def test_idm32_d8192_fanin8_aggregation_traced(paper_keys):
    """The cheaper aggregation (one bootstrap per 8 inputs): the same
    plaintext answer with 32 x 1,171 instead of 32 x 8,191 aggregation
    bootstraps, every traced gate bit-identical to the oracle."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    D, g = 8192, 8
    w, x, ids, pay = idm_inputs(s, D)
    agg = np.zeros((32, 631), dtype=np.uint32)
    vp.velopir_profile(ctx.h, True)
    vp.velopir_trace_start(ctx.h, TRACE_SEED + 1, 32, 200, 4096)
    vp.velopir_query_batch(ctx.h, [vp.make_query(vp.VP_QUERY_IDM, x, ids, D, agg, id_bits=32, payload=pay,
                                                 payload_bits=32, agg_fanin=g)])
    recs = vp.velopir_trace_stop(ctx.h, 4096)
    _, rotations, _ = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_BLIND_ROTATE)
    vp.velopir_profile(ctx.h, False)
    assert rotations == 31 * D + 32 * fanin_nodes(D, g) == 31 * D + 32 * 1171
    got = vp.velopir_client_decrypt_bits(s, agg)
    assert sum(int(b) << j for j, b in enumerate(got)) == int(pay[w["planted"]])
    assert len(recs) < 4096
    assert (recs["nin"] > 2).any(), "no multi-input sum was traced"
    check_trace(paper_keys, recs, 1024)


def test_idm_fanin_whole_circuit_equals_oracle(paper_keys):
    """Whole circuit, small D, every fan-in form: the ciphertexts equal the
    oracle's fan-in tree from the query's own inputs."""
    ctx, s = gpu_ctx()
    D = 11
    w = synth.idm_workload(D, 8, payload=True, substream=23)
    x = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["query"]], 8)[0], synth.lwe_material(8, substream=24))
    ids, pay = w["ids"].astype(np.uint32), w["payload"].astype(np.uint32)
    for g in (3, 4, 8):
        out = np.zeros((32, 631), dtype=np.uint32)
        vp.velopir_query_batch(ctx.h, [vp.make_query(vp.VP_QUERY_IDM, x, ids, D, out, id_bits=8, payload=pay,
                                                     payload_bits=32, agg_fanin=g)])
        assert np.array_equal(out, oracle.idm_payload(paper_keys, x, ids, pay, 32, fanin=g)), g


def test_cov_12_uneven_queries_one_graph_traced(paper_keys):
    """Config 4's shape at 12 queries: D log-uniform in [256, 16,384], all
    layers of all queries packed into one program captured in a CUDA graph."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    vp.velopir_autotune(ctx.h)
    sizes = synth.log_uniform_sizes(12, 256, 16384, substream=19)
    qs, recs_q = [], []
    for q, D in enumerate(sizes):
        w = synth.cov_workload(int(D), substream=300 + q)
        cell = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["cell"]], 32)[0],
                                              synth.lwe_material(32, substream=400 + q))
        cells = w["cells"].astype(np.uint32)
        out = np.zeros((int(D), 631), dtype=np.uint32)
        qs.append((w, cell, cells, out))
        recs_q.append(vp.make_query(vp.VP_QUERY_COV, cell, cells, int(D), out))
    vp.velopir_trace_start(ctx.h, TRACE_SEED + 2, 8, 270, 16384)   # >= 1,137,793 / 270 = 4,215 gates
    vp.velopir_query_batch(ctx.h, recs_q, use_graph=True)
    recs = vp.velopir_trace_stop(ctx.h, 16384)
    assert len(recs) < 16384
    for q, (w, cell, cells, out) in enumerate(qs):
        bits = vp.velopir_client_decrypt_bits(s, out)
        assert np.array_equal(bits, (cells == w["cell"]).astype(np.uint32)), q
    for q in (0, 5, 11):
        w, cell, cells, out = qs[q]
        sample = sorted({0, len(cells) - 1, w["planted"]})
        assert np.array_equal(out[sample], oracle.cov_batch(paper_keys, cell, cells[sample]))
    check_trace(paper_keys, recs, 4096)
