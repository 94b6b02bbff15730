"""Client-side preprocessing on the GPU (velopir_gpu_*), through the C ABI,
against the oracle bit for bit: the cloud key of Section 2.2 KeyGen (BK and
KSK), Enc with Ecd, Alg. PubKeyGen and Alg. ServerEnc, with host and device
buffers; a key generated and kept on the device loads into a context whose
bootstrapped gates equal the oracle's."""
import numpy as np
import pytest

import oracle
from gpu_common import gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


_KM = {}


def _km():
    """The cloud key's random numbers from the master seed (generated once)."""
    if not _KM:
        _KM["km"] = synth.key_material()
    return _KM["km"]


def test_gpu_keygen_host_buffers_equals_oracle(paper_keys):
    ctx, _ = gpu_ctx()
    km = _km()
    bk = np.full(vp.BK_WORDS, 0xDEADBEEF, dtype=np.uint32)
    ksk = np.full(vp.KSK_WORDS, 0xDEADBEEF, dtype=np.uint32)
    vp.velopir_gpu_keygen(ctx.h, km, bk, ksk)
    assert np.array_equal(bk, paper_keys.bk.reshape(-1))
    assert np.array_equal(ksk, paper_keys.ksk.reshape(-1))


def test_gpu_keygen_on_device_loads_and_bootstraps_like_the_oracle(paper_keys):
    """Key material in, key out, all in device memory; the key goes straight
    into a new context (device-to-device) and its gates equal the oracle's."""
    import torch
    gpu_ctx()
    km = _km()
    dev = type("Km", (), {k: _dev(getattr(km, k)) for k in ("s", "K", "bk_a", "bk_e", "ksk_a", "ksk_e")})
    bk = torch.zeros(vp.BK_WORDS, dtype=torch.int32, device="cuda")
    ksk = torch.zeros(vp.KSK_WORDS, dtype=torch.int32, device="cuda")
    ctx = vp.Context(0)
    try:
        vp.velopir_gpu_keygen(ctx.h, dev, bk, ksk)
        assert np.array_equal(_host(bk), paper_keys.bk.reshape(-1))
        assert np.array_equal(_host(ksk), paper_keys.ksk.reshape(-1))
        vp.velopir_load_cloud_key(ctx.h, bk, ksk)
        vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
        bits = synth.Stream(41, 2, 3).bits(2 * 19)
        ct = oracle.encrypt_bits(paper_keys.s, bits, synth.lwe_material(2 * 19, seed=41)).reshape(19, 2, 631)
        out = np.zeros((19, 631), dtype=np.uint32)
        vp.velopir_bootstrap_batch(ctx.h, vp.VP_NAND, ct, out, 19)
        assert np.array_equal(out, oracle.gate_batch(paper_keys, vp.VP_NAND, ct))
    finally:
        ctx.close()


@pytest.mark.parametrize("count", [1, 37, 5000])
def test_gpu_encrypt_bits_equals_oracle(paper_keys, count):
    ctx, s = gpu_ctx()
    bits = synth.Stream(43, 2, count).bits(count)
    lm = synth.lwe_material(count, seed=43 + count)
    host = np.zeros((count, 631), dtype=np.uint32)
    vp.velopir_gpu_encrypt_bits(ctx.h, s, bits, lm.a, lm.e, host)
    want = oracle.encrypt_bits(paper_keys.s, bits, lm)
    assert np.array_equal(host, want)
    import torch
    d = torch.zeros((count, 631), dtype=torch.int32, device="cuda")
    vp.velopir_gpu_encrypt_bits(ctx.h, _dev(s), _dev(bits), _dev(lm.a), _dev(lm.e), d)
    assert np.array_equal(_host(d), want)
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, host), bits)


def test_gpu_pubkeygen_and_server_encrypt_equal_the_oracle(paper_keys):
    """Alg. PubKeyGen then Alg. ServerEnc over a 500-entry 32-bit database
    (16,000 bits) on the device; every ciphertext equals the oracle's, and
    decrypts to its database bit."""
    import torch
    ctx, s = gpu_ctx()
    D, w = 500, 32
    vals = synth.Stream(47, synth.STREAM_DB, 0).torus(D)
    bits = synth.value_bits(vals, w).reshape(-1).astype(np.uint32)
    lm = synth.lwe_material(bits.size, seed=47, stream=synth.STREAM_PUBKEY)
    pk = torch.zeros((bits.size, 631), dtype=torch.int32, device="cuda")
    vp.velopir_gpu_pubkeygen(ctx.h, _dev(s), _dev(lm.a), _dev(lm.e), pk)
    want_pk = oracle.encrypt_mu(paper_keys.s, lm.a, lm.e, np.zeros(bits.size, dtype=np.uint32))
    assert np.array_equal(_host(pk), want_pk)
    ct = torch.zeros_like(pk)
    vp.velopir_gpu_server_encrypt(ctx.h, pk, _dev(bits), ct)
    want = oracle.server_encrypt(want_pk, bits)
    assert np.array_equal(_host(ct), want)
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, _host(ct)), bits)
    # host buffers, and the host client library agrees
    host_pk = np.zeros((64, 631), dtype=np.uint32)
    sub = synth.lwe_material(64, seed=48, stream=synth.STREAM_PUBKEY)
    vp.velopir_gpu_pubkeygen(ctx.h, s, sub.a, sub.e, host_pk)
    assert np.array_equal(host_pk, vp.velopir_client_pubkeygen(s, sub))
    host_ct = np.zeros_like(host_pk)
    vp.velopir_gpu_server_encrypt(ctx.h, host_pk, bits[:64], host_ct)
    assert np.array_equal(host_ct, oracle.server_encrypt(host_pk, bits[:64]))


def test_gpu_client_bad_arguments_and_empty_calls():
    ctx, s = gpu_ctx()
    km = _km()
    bk = np.zeros(vp.BK_WORDS, dtype=np.uint32)
    ksk = np.zeros(vp.KSK_WORDS, dtype=np.uint32)
    with pytest.raises(vp.VelopirError, match="ERR_ARG"):
        vp.velopir_gpu_keygen(ctx.h, km, bk, ksk, params=vp.Params(500, 1024, 1, 3, 7, 8, 2))
    empty = np.zeros((0, 631), dtype=np.uint32)
    vp.velopir_gpu_encrypt_bits(ctx.h, s, np.zeros(0, np.uint32), np.zeros((0, 630), np.uint32),
                                np.zeros(0, np.uint32), empty)
    vp.velopir_gpu_server_encrypt(ctx.h, empty, np.zeros(0, np.uint32), empty)
    rc = vp.lib().velopir_gpu_pubkeygen(ctx.h, None, None, None, 4, None)
    assert rc == vp.ERRORS_BY_NAME["ERR_ARG"]
    rc = vp.lib().velopir_gpu_server_encrypt(ctx.h, None, None, (1 << 24) + 1, None)
    assert rc == vp.ERRORS_BY_NAME["ERR_ARG"]
