"""The tensor-core path (VP_PATH_TENSOR_F16: the dense external product on
tcgen05.mma kind::f16 with exact fp16 limbs) through the C ABI: ciphertexts
bit-identical to the oracle and to the exact NTT path, for one- and
two-rotation gates, a batch spanning several 128-bootstrap tiles with a
ragged tail, and a whole circuit."""
import numpy as np
import pytest

import oracle
from gpu_common import encrypt_value_bits, gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def _inputs(s, count, arity, seed):
    bits = synth.Stream(seed, 2, 13).bits(count * arity)
    return vp.velopir_client_encrypt_bits(s, bits, synth.lwe_material(count * arity, seed=seed)).reshape(
        count, arity, 631)


@pytest.fixture()
def tensor_ctx():
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_TENSOR_F16)
    try:
        yield ctx, s
    finally:
        vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)


@pytest.mark.parametrize("gate, count, arity", [(vp.VP_AND, 5, 2), (vp.VP_XNOR, 37, 2), (vp.VP_MUX, 11, 3)])
def test_tensor_path_equals_oracle(paper_keys, tensor_ctx, gate, count, arity):
    ctx, s = tensor_ctx
    ct = _inputs(s, count, arity, 1300 + gate)
    out = np.zeros((count, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, gate, ct, out, count)
    assert np.array_equal(out, oracle.gate_batch(paper_keys, gate, ct))


def test_tensor_path_equals_ntt_on_several_tiles(paper_keys, tensor_ctx):
    """300 gates: three 128-bootstrap tiles, the last one ragged."""
    ctx, s = tensor_ctx
    n = 300
    ct = _inputs(s, n, 2, 1310)
    got = np.zeros((n, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_ORYN, ct, got, n)
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    want = np.zeros_like(got)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_ORYN, ct, want, n)
    assert np.array_equal(got, want)
    pick = np.array([0, 127, 128, 255, 256, n - 1])
    assert np.array_equal(got[pick], oracle.gate_batch(paper_keys, vp.VP_ORYN, ct[pick]))


def test_tensor_path_whole_circuit(paper_keys, tensor_ctx):
    ctx, s = tensor_ctx
    w = synth.idm_workload(4, 8)
    x = encrypt_value_bits(s, w["query"], 8, 508)
    ids = w["ids"].astype(np.uint32)
    out = np.zeros((4, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 8, ids, 4, None, 0, out)
    assert np.array_equal(out, oracle.idm_batch(paper_keys, x, ids))
