"""GPU parity of the encrypted-database circuits (Section 3.2's protocol:
every database bit is a ServerEnc ciphertext) against the oracle, bit for
bit, through the C ABI; plus decryption against the plaintext predicates at
the paper's interval precision (l_I = 16)."""
import numpy as np
import pytest

import oracle
from gpu_common import encrypt_value_bits, gpu_ctx
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def server_enc(s, values, width, seed):
    """Alg. PubKeyGen + ServerEnc of plaintext values (LSB first), as the
    library's client and server code compute them: [len(values)][width][631]."""
    bits = synth.value_bits(np.asarray(values, dtype=np.uint64), width)
    pk = vp.velopir_client_pubkeygen(s, synth.lwe_material(bits.size, seed=seed, stream=synth.STREAM_PUBKEY))
    return vp.velopir_server_encrypt(pk, bits.reshape(-1)).reshape(len(values), width, 631)


def test_intv_encdb_matches_oracle(paper_keys):
    ctx, s = gpu_ctx()
    l = 4
    x, y = 9, 6
    rects = np.array([[9, 10, 6, 7], [0, 9, 0, 15], [3, 12, 2, 8]], dtype=np.uint32)
    cx, cy = encrypt_value_bits(s, x, l, 900), encrypt_value_bits(s, y, l, 901)
    enc = server_enc(s, rects.reshape(-1), l, 902).reshape(3, 4, l, 631)
    out = np.zeros((3, 631), dtype=np.uint32)
    vp.velopir_interval_query_encdb(ctx.h, cx, cy, l, enc, 3, None, 0, out)
    v = oracle.intv_enc_batch(paper_keys, cx, cy, enc)
    assert np.array_equal(out, v)
    assert list(vp.velopir_client_decrypt_bits(s, out)) == [1, 0, 1]
    # with 2-bit payloads: the XOR of the payloads of entries 0 and 2
    P = server_enc(s, [1, 2, 3], 2, 903)
    agg = np.zeros((2, 631), dtype=np.uint32)
    vp.velopir_interval_query_encdb(ctx.h, cx, cy, l, enc, 3, P, 2, agg)
    assert np.array_equal(agg, oracle.aggregate_enc(paper_keys, v, P))
    assert list(vp.velopir_client_decrypt_bits(s, agg)) == [0, 1]


def test_cov_encdb_matches_oracle(paper_keys):
    ctx, s = gpu_ctx()
    w = 3
    q = (5 << w) | 2
    cells = np.array([q, (5 << w) | 3, (4 << w) | 2, 0], dtype=np.uint32)
    cq = encrypt_value_bits(s, q, 2 * w, 910)
    enc = server_enc(s, cells, 2 * w, 911)
    out = np.zeros((4, 631), dtype=np.uint32)
    vp.velopir_coordinate_query_encdb(ctx.h, cq, w, enc, 4, None, 0, out)
    assert np.array_equal(out, oracle.cov_enc_batch(paper_keys, cq, enc, w))
    assert list(vp.velopir_client_decrypt_bits(s, out)) == [1, 0, 0, 0]


def test_idm_encdb_payload_matches_oracle(paper_keys):
    ctx, s = gpu_ctx()
    l, lS = 4, 3
    ids = np.array([5, 12, 7], dtype=np.uint32)
    pay = np.array([3, 6, 5], dtype=np.uint32)
    xq = encrypt_value_bits(s, 12, l, 920)
    E = server_enc(s, ids, l, 921)
    P = server_enc(s, pay, lS, 922)
    match = np.zeros((3, 631), dtype=np.uint32)
    vp.velopir_id_match_encdb(ctx.h, xq, l, E, 3, None, 0, match)
    assert np.array_equal(match, oracle.idm_enc_batch(paper_keys, xq, E))
    agg = np.zeros((lS, 631), dtype=np.uint32)
    vp.velopir_id_match_encdb(ctx.h, xq, l, E, 3, P, lS, agg)
    assert np.array_equal(agg, oracle.idm_enc_payload(paper_keys, xq, E, P))
    assert list(vp.velopir_client_decrypt_bits(s, agg)) == [0, 1, 1]


def test_intv_encdb_paper_precision_device_buffers(paper_keys):
    """l_I = 16 (the paper's datasets), D = 96 from device memory: every
    output decrypts to the predicate; one entry is recomputed by the oracle."""
    import torch
    ctx, s = gpu_ctx()
    l, D = 16, 96
    st = synth.Stream(synth.MASTER_SEED, synth.STREAM_DB, 77)
    x, y = (int(v) & 0xFFFF for v in st.words(2))
    u = (st.words(4 * D) & np.uint32(0xFFFF)).reshape(D, 4).astype(np.int64)
    lo, hi = np.minimum(u[:, [0, 2]], u[:, [1, 3]]), np.maximum(u[:, [0, 2]], u[:, [1, 3]]) + 1
    lo[::4, 0], hi[::4, 0], lo[::4, 1], hi[::4, 1] = x, x + 1, max(0, y - 3), y + 1
    hi = np.minimum(hi, 0xFFFF)
    rects = np.stack([lo[:, 0], hi[:, 0], lo[:, 1], hi[:, 1]], axis=1).astype(np.uint32)
    cx, cy = encrypt_value_bits(s, x, l, 930), encrypt_value_bits(s, y, l, 931)
    enc = server_enc(s, rects.reshape(-1), l, 932).reshape(D, 4, l, 631)
    dout = torch.zeros((D, 631), dtype=torch.int32, device="cuda")
    vp.velopir_interval_query_encdb(ctx.h, torch.from_numpy(cx.view(np.int32)).cuda(),
                                    torch.from_numpy(cy.view(np.int32)).cuda(), l,
                                    torch.from_numpy(enc.view(np.int32)).cuda(), D, None, 0, dout)
    out = dout.cpu().numpy().view(np.uint32)
    r = rects.astype(np.int64)
    want = ((r[:, 0] <= x) & (x < r[:, 1]) & (r[:, 2] <= y) & (y < r[:, 3])).astype(np.uint32)
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, out), want) and want.sum() > 0
    assert np.array_equal(out[:1], oracle.intv_enc_batch(paper_keys, cx, cy, enc[:1]))


def test_encdb_bad_arguments():
    ctx, s = gpu_ctx()
    z = np.zeros((4, 631), dtype=np.uint32)
    with pytest.raises(vp.VelopirError):
        vp.velopir_interval_query_encdb(ctx.h, z, z, 0, z, 1, None, 0, z)
    with pytest.raises(vp.VelopirError):
        vp.velopir_coordinate_query_encdb(ctx.h, z, 17, z, 1, None, 0, z)
    with pytest.raises(vp.VelopirError):
        vp.velopir_coordinate_query_encdb(ctx.h, z, 4, z, 1, z, 4097, z)
    with pytest.raises(vp.VelopirError):
        vp.velopir_id_match_encdb(ctx.h, z, 33, z, 1, None, 0, z)
    vp.velopir_id_match_encdb(ctx.h, z, 4, z, 0, None, 0, z)   # D = 0 is a no-op


@pytest.mark.parametrize("fanin", [4, 8])
def test_encdb_fanin_aggregation_matches_oracle(paper_keys, fanin):
    """velopir_set_encdb_fanin: the HomBitwiseAND results of D = 11 entries
    XOR-aggregated by the fan-in-g tree, bit-identical to the oracle's
    composition (match bits, ANDs, homsum_tree_fanin), for IdM and CoV."""
    ctx, s = gpu_ctx()
    l, lS, D = 6, 5, 11
    rng = np.random.default_rng(940 + fanin)
    ids = rng.choice(1 << l, size=D, replace=False).astype(np.uint32)
    pay = rng.integers(0, 1 << lS, size=D, dtype=np.uint64).astype(np.uint32)
    xq = encrypt_value_bits(s, int(ids[4]), l, 941)
    E = server_enc(s, ids, l, 942)
    P = server_enc(s, pay, lS, 943)
    vp.velopir_set_encdb_fanin(ctx.h, fanin)
    try:
        agg = np.zeros((lS, 631), dtype=np.uint32)
        vp.velopir_id_match_encdb(ctx.h, xq, l, E, D, P, lS, agg)
        w = 3
        cells = (ids & np.uint32(0x3F)).astype(np.uint32)
        cells[::3] = cells[1]
        cq = encrypt_value_bits(s, int(cells[1]), 2 * w, 944)
        C = server_enc(s, cells, 2 * w, 945)
        cagg = np.zeros((lS, 631), dtype=np.uint32)
        vp.velopir_coordinate_query_encdb(ctx.h, cq, w, C, D, P, lS, cagg)
    finally:
        vp.velopir_set_encdb_fanin(ctx.h, 0)
    m = oracle.idm_enc_batch(paper_keys, xq, E)
    assert np.array_equal(agg, oracle.aggregate_enc(paper_keys, m, P, fanin=fanin))
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, agg), synth.value_bits([pay[4]], lS)[0])
    v = oracle.cov_enc_batch(paper_keys, cq, C, w)
    assert np.array_equal(cagg, oracle.aggregate_enc(paper_keys, v, P, fanin=fanin))
    want = np.bitwise_xor.reduce(pay[cells == cells[1]])
    assert np.array_equal(vp.velopir_client_decrypt_bits(s, cagg), synth.value_bits([want], lS)[0])
    with pytest.raises(vp.VelopirError):
        vp.velopir_set_encdb_fanin(ctx.h, 9)
