"""The paper's Table 4 workload shapes (synthetic stand-ins with its M, l_I
and l_S) through the full encrypted-database protocol on the GPU: Alg.
PubKeyGen + ServerEnc, validation, HomBitwiseAND with the encrypted payload
and the HomSum XOR tree.

  * gdacs CoV (M = 9, l_S = 16, 839 bootstraps): the whole circuit equals the
    oracle's from the query's own ciphertexts;
  * covid-usa IntV (M = 58, l_S = 22, 13,840 bootstraps) and weather-usa IdM
    (M = 304, l_S = 128, 87,120 bootstraps; 53,968 with the fan-in-8 XOR
    tree): traced gates of every launch recomputed by the oracle, and the
    aggregate decrypts to the XOR of the valid entries' payloads."""
import numpy as np
import pytest

import oracle
from gpu_common import check_trace, gpu_ctx
from paper_2506_12761_gb300 import config_bench as cb
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def _case(name, mode):
    return next(k for k, row in enumerate(cb.PAPER4) if row[0] == name and row[1] == mode)


def test_gdacs_cov_whole_protocol_equals_oracle(paper_keys):
    ctx, s = gpu_ctx()
    c = cb.paper4_case(s, _case("gdacs", "CoV"))
    out = np.zeros((c["lS"], 631), dtype=np.uint32)
    cb.paper4_run(ctx.h, c, out)
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, out), c["want"])
    v = oracle.cov_enc_batch(paper_keys, c["cq"], c["enc"], c["l"])
    assert np.array_equal(out, oracle.aggregate_enc(paper_keys, v, c["P"]))


@pytest.mark.parametrize("name, mode, one_in, fanin", [("covid-usa", "IntV", 8, 2), ("weather-usa", "IdM", 60, 2),
                                                       ("weather-usa", "IdM", 40, 8)])
def test_paper_shape_traced(paper_keys, name, mode, one_in, fanin):
    ctx, s = gpu_ctx()
    c = cb.paper4_case(s, _case(name, mode))
    out = np.zeros((c["lS"], 631), dtype=np.uint32)
    vp.velopir_set_encdb_fanin(ctx.h, fanin)
    vp.velopir_trace_start(ctx.h, 4242, 8, one_in, 4096)
    try:
        cb.paper4_run(ctx.h, c, out)
    finally:
        recs = vp.velopir_trace_stop(ctx.h, 4096)
        vp.velopir_set_encdb_fanin(ctx.h, 0)
    assert len(recs) < 4096
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, out), c["want"])
    assert (recs["nrot"] == 2).any() == (mode == "IntV")   # the comparators' MUXes
    assert (recs["nin"] == fanin).any() if fanin > 2 else (recs["nin"] <= 3).all()
    check_trace(paper_keys, recs, 800)
