"""velopir_bootstrap_batch_noalloc, the allocation-free entry point, through
the C ABI: on two calls in a row its ciphertexts equal those of
velopir_bootstrap_batch (the tolerance of every parity test here: zero bits).

It exists for callers that cannot allocate device memory while they run (a
server that reserved its HBM at start-up, a hard memory cap, a latency-critical
loop where cudaMalloc/cudaFree would stall the device).  This file is named so
that pytest collects it last; it passes alone in a fresh process (it sets up
its own context) and after the other tests."""
import numpy as np
import pytest

from gpu_common import gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def _inputs(s, count, arity, seed):
    import torch
    bits = synth.Stream(seed, 2, 11).bits(count * arity)
    ct = vp.velopir_client_encrypt_bits(s, bits, synth.lwe_material(count * arity, seed=seed))
    return torch.from_numpy(ct.reshape(count, arity, 631).view(np.int32)).cuda()


def test_noalloc_equals_batched_on_two_calls_in_a_row():
    import torch
    ctx, s = gpu_ctx()
    calls = [(vp.VP_AND, 37, 2, 1201), (vp.VP_MUX, 11, 3, 1202)]
    for gate, count, arity, seed in calls:
        din = _inputs(s, count, arity, seed)
        want = torch.zeros((count, 631), dtype=torch.int32, device="cuda")
        got = torch.full((count, 631), -1, dtype=torch.int32, device="cuda")
        vp.velopir_bootstrap_batch(ctx.h, gate, din, want, count)
        vp.velopir_bootstrap_batch_noalloc(ctx.h, gate, din, got, count)
        assert torch.equal(got, want)


def test_noalloc_limits():
    import torch
    ctx, s = gpu_ctx()
    n = vp.NOALLOC_MAX_GATES
    din = _inputs(s, n, 2, 1203)
    out = torch.zeros((n, 631), dtype=torch.int32, device="cuda")
    vp.velopir_bootstrap_batch_noalloc(ctx.h, vp.VP_XOR, din, out, n)          # the maximum is accepted
    ref = torch.zeros_like(out)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_XOR, din, ref, n)
    assert torch.equal(out, ref)
    with pytest.raises(vp.VelopirError, match="VELOPIR_NOALLOC_MAX_GATES"):
        vp.velopir_bootstrap_batch_noalloc(ctx.h, vp.VP_XOR, din, out, n + 1)
    host = np.zeros((1, 2, 631), dtype=np.uint32)
    with pytest.raises(vp.VelopirError, match="device memory"):
        vp.velopir_bootstrap_batch_noalloc(ctx.h, vp.VP_AND, host, out, 1)
