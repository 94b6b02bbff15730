"""velopir_bootstrap_batch_noalloc, the allocation-free entry point, through
the C ABI: on two calls in a row its ciphertexts equal the oracle's gates and
those of velopir_bootstrap_batch (the tolerance of every parity test here:
zero bits), on the NTT path and on the dense path it takes before a
context's transformed key exists, and at the size limit for both one- and
two-rotation gates.

It exists for callers that cannot allocate device memory while they run (a
server that reserved its HBM at start-up, a hard memory cap, a latency-critical
loop where cudaMalloc/cudaFree would stall the device).  This file is named so
that pytest collects it last; it passes alone in a fresh process (it sets up
its own context) and after the other tests."""
import numpy as np
import pytest

import oracle
from gpu_common import _state, gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def _inputs(s, count, arity, seed):
    bits = synth.Stream(seed, 2, 11).bits(count * arity)
    return vp.velopir_client_encrypt_bits(s, bits, synth.lwe_material(count * arity, seed=seed)).reshape(
        count, arity, 631)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def test_noalloc_equals_oracle_and_batched_on_two_calls_in_a_row(paper_keys):
    import torch
    ctx, s = gpu_ctx()
    calls = [(vp.VP_AND, 37, 2, 1201), (vp.VP_MUX, 11, 3, 1202)]
    for gate, count, arity, seed in calls:
        ct = _inputs(s, count, arity, seed)
        din = _dev(ct)
        want = torch.zeros((count, 631), dtype=torch.int32, device="cuda")
        got = torch.full((count, 631), -1, dtype=torch.int32, device="cuda")
        vp.velopir_bootstrap_batch(ctx.h, gate, din, want, count)
        vp.velopir_bootstrap_batch_noalloc(ctx.h, gate, din, got, count)
        assert torch.equal(got, want)
        assert np.array_equal(_host(got), oracle.gate_batch(paper_keys, gate, ct))


def test_noalloc_first_call_on_a_fresh_context_takes_the_dense_path(paper_keys):
    """Before any other bootstrap on a context, the transformed NTT key does
    not exist yet and the call runs the dense path: same bits as the oracle."""
    import torch
    gpu_ctx()
    ctx = vp.Context(0)
    try:
        vp.velopir_load_cloud_key(ctx.h, _state["bk"], _state["ksk"])
        vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
        ct = _inputs(_state["s"], 9, 2, 1204)
        out = torch.zeros((9, 631), dtype=torch.int32, device="cuda")
        vp.velopir_bootstrap_batch_noalloc(ctx.h, vp.VP_ORNY, _dev(ct), out, 9)
        assert np.array_equal(_host(out), oracle.gate_batch(paper_keys, vp.VP_ORNY, ct))
    finally:
        ctx.close()


@pytest.mark.parametrize("gate, arity", [(vp.VP_XOR, 2), (vp.VP_MUX, 3)])
def test_noalloc_at_the_limit(paper_keys, gate, arity):
    """count = VELOPIR_NOALLOC_MAX_GATES (for MUX: 512 rotations, the whole
    scratch array) equals velopir_bootstrap_batch, and sampled gates equal
    the oracle; one more gate is refused, and so is host memory."""
    import torch
    ctx, s = gpu_ctx()
    n = vp.NOALLOC_MAX_GATES
    ct = _inputs(s, n, arity, 1203 + arity)
    din = _dev(ct)
    out = torch.zeros((n, 631), dtype=torch.int32, device="cuda")
    vp.velopir_bootstrap_batch_noalloc(ctx.h, gate, din, out, n)          # the maximum is accepted
    ref = torch.zeros_like(out)
    vp.velopir_bootstrap_batch(ctx.h, gate, din, ref, n)
    assert torch.equal(out, ref)
    pick = np.array([0, 1, 77, 128, 200, n - 1])
    assert np.array_equal(_host(out)[pick], oracle.gate_batch(paper_keys, gate, ct[pick]))
    with pytest.raises(vp.VelopirError, match="VELOPIR_NOALLOC_MAX_GATES"):
        vp.velopir_bootstrap_batch_noalloc(ctx.h, gate, din, out, n + 1)
    host = np.zeros((1, arity, 631), dtype=np.uint32)
    with pytest.raises(vp.VelopirError, match="device memory"):
        vp.velopir_bootstrap_batch_noalloc(ctx.h, gate, host, out, 1)
