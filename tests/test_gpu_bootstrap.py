"""GPU parity of velopir_bootstrap_batch / _plain against the oracle, bit for
bit, through the C ABI (every path, every gate, ragged batch sizes)."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu
PATHS = [vp.VP_PATH_INT32_DENSE, vp.VP_PATH_NTT]


def random_inputs(s, count, arity, seed):
    bits = synth.Stream(seed, 2, 5).bits(count * arity)
    ct = vp.velopir_client_encrypt_bits(s, bits, synth.lwe_material(count * arity, seed=seed))
    return ct.reshape(count, arity, 631), bits.reshape(count, arity)


@pytest.mark.parametrize("path", PATHS)
def test_and_batch_spans_tiles_with_ragged_tail(path, paper_keys):
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, path)
    inp, bits = random_inputs(s, 19, 2, seed=31)
    out = np.zeros((19, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_AND, inp, out, 19)
    want = oracle.gate_batch(paper_keys, oracle.AND, inp)
    assert np.array_equal(out, want)
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, out), bits[:, 0] & bits[:, 1])


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("gate", list(range(10)))
def test_every_binary_gate(path, gate, paper_keys):
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, path)
    inp, _ = random_inputs(s, 4, 2, seed=40 + gate)
    out = np.zeros((4, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, gate, inp, out, 4)
    assert np.array_equal(out, oracle.gate_batch(paper_keys, gate, inp))


@pytest.mark.parametrize("path", PATHS)
def test_mux_and_device_buffers(path, paper_keys):
    import torch
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, path)
    inp, bits = random_inputs(s, 9, 3, seed=60)
    din = torch.from_numpy(inp.view(np.int32)).cuda()
    dout = torch.zeros((9, 631), dtype=torch.int32, device="cuda")
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_MUX, din, dout, 9)
    out = dout.cpu().numpy().view(np.uint32)
    assert np.array_equal(out, oracle.gate_batch(paper_keys, oracle.MUX, inp))
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, out), np.where(bits[:, 0] == 1, bits[:, 1], bits[:, 2]))


@pytest.mark.parametrize("path", PATHS)
def test_plain_equals_batched(path, paper_keys):
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, path)
    inp, _ = random_inputs(s, 3, 2, seed=70)
    a = np.zeros((3, 631), dtype=np.uint32)
    b = np.zeros((3, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_XOR, inp, a, 3)
    vp.velopir_bootstrap_plain(ctx.h, vp.VP_XOR, inp, b, 3)
    assert np.array_equal(a, b) and np.array_equal(a, oracle.gate_batch(paper_keys, oracle.XOR, inp))


def test_empty_and_bad_arguments():
    ctx, s = gpu_ctx()
    z = np.zeros((1, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_AND, z, z, 0)      # count 0: no-op
    with pytest.raises(vp.VelopirError):
        vp.velopir_bootstrap_batch(ctx.h, 99, z, z, 1)
    with pytest.raises(vp.VelopirError):
        vp.velopir_set_path(ctx.h, 7)


@pytest.mark.parametrize("path", PATHS)
def test_trivial_inputs_take_no_rotation_steps(path, paper_keys):
    """A trivial input (zero mask) rotates by abar_i = 0 at every step."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, path)
    inp = np.zeros((2, 2, 631), dtype=np.uint32)
    inp[0, :, 630] = 1 << 29
    inp[1, 0, 630] = (1 << 32) - (1 << 29)
    out = np.zeros((2, 631), dtype=np.uint32)
    vp.velopir_bootstrap_batch(ctx.h, vp.VP_AND, inp, out, 2)
    assert np.array_equal(out, oracle.gate_batch(paper_keys, oracle.AND, inp))


def test_paths_agree_on_a_larger_batch():
    """The dense and NTT paths give identical bits on a batch spanning many CTAs."""
    ctx, s = gpu_ctx()
    inp, bits = random_inputs(s, 157, 2, seed=80)
    outs = []
    for path in PATHS:
        vp.velopir_set_path(ctx.h, path)
        o = np.zeros((157, 631), dtype=np.uint32)
        vp.velopir_bootstrap_batch(ctx.h, vp.VP_ORYN, inp, o, 157)
        outs.append(o)
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, outs[1]), bits[:, 0] | (1 - bits[:, 1]))


def test_autotuned_shapes_keep_parity(paper_keys):
    """After the autotuner has timed every tile shape, batches of sizes that
    favour different shapes still match the oracle bit for bit."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    waves = vp.velopir_autotune(ctx.h)
    assert len(waves) == len(vp.NTT_TILE_SHAPES) and all(w > 0 for w in waves)
    shapes = {vp.velopir_tuned_shape(ctx.h, n) for n in (152 * 4, 152 * 5, 152 * 6, 152 * 7, 1000, 4096)}
    assert shapes <= set(vp.NTT_TILE_SHAPES)
    for count, seed in ((13, 90), (29, 91)):
        inp, _ = random_inputs(s, count, 2, seed=seed)
        out = np.zeros((count, 631), dtype=np.uint32)
        vp.velopir_bootstrap_batch(ctx.h, vp.VP_NAND, inp, out, count)
        assert np.array_equal(out, oracle.gate_batch(paper_keys, oracle.NAND, inp))
