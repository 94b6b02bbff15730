"""Pins of the oracle's encrypted-database functions (Section 3.2's
PubKeyGen/ServerEnc preprocessing and the circuits with both operands
encrypted), by decryption against plaintext predicates at the toy parameter
set (n = 32, N = 256) -- exhaustive where the input space is small -- and of
the library's client PubKeyGen/ServerEnc against the oracle bit for bit."""
import itertools
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
from paper_2506_12761_gb300 import synth


def bits_of(v, l):
    return [(v >> i) & 1 for i in range(l)]


def enc_value(keys, v, l, seed):
    return oracle.encrypt_bits(keys.s, bits_of(v, l), synth.lwe_material(l, keys.P.n, seed=seed))


def server_enc_value(keys, v, l, seed):
    """A database value as Alg. ServerEnc encrypts it: public-key ciphertexts
    (encryptions of zero, Alg. PubKeyGen) plus the encoded bits."""
    lm = synth.lwe_material(l, keys.P.n, seed=seed, stream=synth.STREAM_PUBKEY)
    pk = oracle.encrypt_mu(keys.s, lm.a, lm.e, np.zeros(l, dtype=np.uint32))
    return oracle.server_encrypt(pk, bits_of(v, l))


def pmap(f, items):
    with ThreadPoolExecutor(8) as ex:
        return list(ex.map(f, items))


def test_server_encrypt_decrypts_to_the_bits(toy_keys):
    bits = [0, 1, 1, 0, 1, 0, 0, 1]
    lm = synth.lwe_material(len(bits), toy_keys.P.n, seed=11, stream=synth.STREAM_PUBKEY)
    pk = oracle.encrypt_mu(toy_keys.s, lm.a, lm.e, np.zeros(len(bits), dtype=np.uint32))
    # an encryption of zero has a phase equal to its noise
    assert np.array_equal(oracle.phase(toy_keys.s, pk), lm.e)
    ct = oracle.server_encrypt(pk, bits)
    assert list(oracle.decrypt_bits(toy_keys.s, ct)) == bits
    # ServerEnc only moves b by +-1/8: the masks are the public key's
    assert np.array_equal(ct[:, :-1], pk[:, :-1])
    assert np.array_equal(ct[:, -1] - pk[:, -1], np.where(np.array(bits) == 1, oracle.MU, (1 << 32) - oracle.MU).astype(np.uint32))


def test_library_pubkeygen_and_server_encrypt_match_the_oracle(paper_keys):
    from paper_2506_12761_gb300 import velopir as vp
    km = synth.key_material()
    lm = synth.lwe_material(40, seed=12, stream=synth.STREAM_PUBKEY)
    pk = vp.velopir_client_pubkeygen(km.s, lm)
    want = oracle.encrypt_mu(paper_keys.s, lm.a, lm.e, np.zeros(40, dtype=np.uint32))
    assert np.array_equal(pk, want)
    bits = synth.Stream(12, 3, 1).bits(40)
    assert np.array_equal(vp.velopir_server_encrypt(pk, bits), oracle.server_encrypt(want, bits))


def test_toy_unsigned_encrypted_comparators_all_pairs(toy_keys):
    l = 3
    a_cts = {v: server_enc_value(toy_keys, v, l, 100 + v) for v in range(1 << l)}
    x_cts = {v: enc_value(toy_keys, v, l, 200 + v) for v in range(1 << l)}
    jobs = list(itertools.product(range(1 << l), repeat=2))

    def run(job):
        a, x = job
        return [int(oracle.decrypt_bits(toy_keys.s, oracle.comp_enc_unsigned(toy_keys, a_cts[a], x_cts[x], strict))[0])
                for strict in (False, True)]

    for (a, x), got in zip(jobs, pmap(run, jobs)):
        assert got == [int(a <= x), int(a < x)], (a, x)


def test_toy_intv_enc(toy_keys):
    l = 4
    x, y = 9, 6
    cx, cy = enc_value(toy_keys, x, l, 300), enc_value(toy_keys, y, l, 301)
    rects = [(9, 10, 6, 7), (0, 9, 0, 15), (10, 15, 0, 15), (0, 15, 7, 8), (3, 12, 2, 8), (8, 9, 5, 6), (9, 15, 6, 15)]
    enc = np.stack([np.stack([server_enc_value(toy_keys, v, l, 400 + 4 * d + k) for k, v in enumerate(r)])
                    for d, r in enumerate(rects)])
    out = oracle.intv_enc_batch(toy_keys, cx, cy, enc)
    want = [int(r[0] <= x < r[1] and r[2] <= y < r[3]) for r in rects]
    assert list(oracle.decrypt_bits(toy_keys.s, out)) == want and 0 < sum(want) < len(want)


def test_toy_cov_enc_all_cells(toy_keys):
    w = 2
    q = (2 << w) | 1
    cq = enc_value(toy_keys, q, 2 * w, 500)
    cells = list(range(1 << (2 * w)))
    enc = np.stack([server_enc_value(toy_keys, c, 2 * w, 600 + c) for c in cells])
    out = oracle.cov_enc_batch(toy_keys, cq, enc, w)
    assert list(oracle.decrypt_bits(toy_keys.s, out)) == [int(c == q) for c in cells]


def test_toy_idm_enc_payload(toy_keys):
    l, lS = 3, 3
    ids = [5, 2, 7, 0, 6]
    pay = [3, 6, 1, 7, 4]
    q = 7
    xq = enc_value(toy_keys, q, l, 700)
    E = np.stack([server_enc_value(toy_keys, v, l, 800 + d) for d, v in enumerate(ids)])
    P = np.stack([server_enc_value(toy_keys, v, lS, 900 + d) for d, v in enumerate(pay)])
    match = oracle.idm_enc_batch(toy_keys, xq, E)
    assert list(oracle.decrypt_bits(toy_keys.s, match)) == [int(i == q) for i in ids]
    agg = oracle.idm_enc_payload(toy_keys, xq, E, P)
    assert list(oracle.decrypt_bits(toy_keys.s, agg)) == bits_of(pay[ids.index(q)], lS)
    miss = oracle.idm_enc_payload(toy_keys, enc_value(toy_keys, 1, l, 701), E, P)
    assert list(oracle.decrypt_bits(toy_keys.s, miss)) == [0] * lS


def test_toy_aggregate_xors_the_valid_payloads(toy_keys):
    """With several valid entries the aggregate is the XOR of their payloads
    (HomSum of the zeroed payloads), including a single entry (no XOR)."""
    lS = 4
    valid = [1, 0, 1, 1, 0, 1, 0]
    pay = [9, 3, 5, 12, 15, 6, 1]
    v = np.stack([server_enc_value(toy_keys, b, 1, 1000 + d)[0] for d, b in enumerate(valid)])
    P = np.stack([server_enc_value(toy_keys, p, lS, 1100 + d) for d, p in enumerate(pay)])
    agg = oracle.aggregate_enc(toy_keys, v, P)
    want = 0
    for b, p in zip(valid, pay):
        want ^= p if b else 0
    assert list(oracle.decrypt_bits(toy_keys.s, agg)) == bits_of(want, lS)
    one = oracle.aggregate_enc(toy_keys, v[:1], P[:1])
    assert list(oracle.decrypt_bits(toy_keys.s, one)) == bits_of(pay[0], lS)
