"""Pins of the oracle's parameters, encoding, key generation, modulus switch
and gadget decomposition against the paper and closed forms."""
from fractions import Fraction

import numpy as np

import oracle
from conftest import read_golden
from paper_2506_12761_gb300 import synth
from test_oracle_poly import kronecker_negacyclic

M32 = (1 << 32) - 1


def test_parameters_match_paper_table():
    g = read_golden("tfhe_params.txt")
    P = oracle.paper_params()
    assert (P.n, P.N, P.l, P.bg_bits, P.ks_t, P.ks_base_bits) == (
        int(g["n"][0]), int(g["N"][0]), int(g["bk_level"][0]), int(g["bk_base_log2"][0]),
        int(g["ks_level"][0]), int(g["ks_base_log2"][0]))
    assert int(g["k"][0]) == 1
    assert synth.SIGMA_KS_LOG2 == int(g["sigma_ks_log2"][0])
    assert synth.SIGMA_BK_LOG2 == int(g["sigma_bk_log2"][0])
    assert synth.PAPER_PARAMS == dict(n=630, N=1024, k=1, l=3, bg_bits=7, ks_t=8, ks_base_bits=2)


def test_encrypt_phase_and_decrypt():
    km = synth.key_material(n=630, N=16, l=1, ks_t=1, ks_base_bits=1)  # only s is used
    lm = synth.lwe_material(64)
    bits = synth.Stream(3, 2, 0).bits(64)
    ct = oracle.encrypt_bits(km.s, bits, lm)
    ph = oracle.phase(km.s, ct)
    mu = np.where(bits != 0, 1 << 29, (1 << 32) - (1 << 29)).astype(np.uint32)
    assert np.array_equal(ph, (mu + lm.e[:64]).astype(np.uint32))   # phase = mu + e exactly
    assert np.array_equal(oracle.decrypt_bits(km.s, ct), bits)
    # Ecd: m -> m/4 - 1/8 (Section 2.2)
    assert (1 << 32) * (Fraction(1, 4) - Fraction(1, 8)) == 1 << 29
    # tie rule: phase 0 decodes as 1
    z = oracle.trivial(630, 0)
    assert oracle.decrypt_bits(km.s, z)[0] == 1


def test_modswitch_is_exact_rounding():
    N = 1024
    rng = np.random.default_rng(3)
    xs = list(rng.integers(0, 1 << 32, 5000, dtype=np.uint64)) + [0, M32, 1 << 20, (1 << 20) - 1,
                                                                    (1 << 21) + (1 << 20), (1 << 31)]
    for x in xs:
        want = int(Fraction(int(x) * 2 * N, 1 << 32) + Fraction(1, 2)) % (2 * N)  # floor(y + 1/2)
        assert oracle.modswitch(int(x), N) == want


def test_decompose_bound_and_range():
    P = oracle.paper_params()
    rng = np.random.default_rng(4)
    xs = list(rng.integers(0, 1 << 32, 20000, dtype=np.uint64))
    xs += [0, M32, 1 << 31, (1 << 10), (1 << 10) - 1, (1 << 11) - 1, 0x7FFFFFFF, 0x80000400]
    for x in xs:
        d = oracle.decompose(P, int(x))
        assert d.min() >= -64 and d.max() <= 63
        rec = sum(int(d[p]) << (32 - 7 * (p + 1)) for p in range(3)) & M32
        err = (rec - int(x)) & M32
        err = err - (1 << 32) if err >= (1 << 31) else err
        assert -(1 << 10) <= err <= (1 << 10)


def test_keygen_rows_decrypt(toy_keys):
    """BK rows are TRLWE encryptions of s_i * h_p on component q; KSK rows
    encrypt v*K_i*2^(32-2(j+1)); both with noise of the stated width."""
    k = toy_keys
    P = k.P
    for i in range(P.n):
        for r in range(2 * P.l):
            p, q = r // 2 + 1, r % 2
            a, b = k.bk[i, r, 0], k.bk[i, r, 1]
            ph = (b.astype(np.int64) - kronecker_negacyclic(a, k.K).astype(np.int64)) & M32
            h = int(k.s[i]) << (32 - 7 * p)
            # phase(row) = e - h*K (q = 0) or e + h (q = 1) in coefficient form
            if q == 1:
                expect = np.zeros(P.N, dtype=np.int64); expect[0] = h
            else:
                expect = (-(h * k.K.astype(np.int64))) & M32
            e = ((ph - expect) & M32).astype(np.uint32).view(np.int32)
            assert np.abs(e).max() < 2 ** 12   # sigma_BK = 2^-25 -> 2^7 units
    for i in range(0, P.N, 37):
        for j in range(P.ks_t):
            for v in range(4):
                row = k.ksk[i, j, v]
                ph = int(oracle.phase(k.s, row)[0])
                want = (v * int(k.K[i]) << (32 - 2 * (j + 1))) & M32
                e = ((ph - want) & M32)
                e = e - (1 << 32) if e >= (1 << 31) else e
                assert abs(e) < 2 ** 22             # sigma_KS = 2^-15 -> 2^17 units
