"""Pins of the oracle's blind rotation, sample extraction, key switch, gates
and noise against closed forms, invariants, truth tables and tfhe-2's bound."""
import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2506_12761_gb300 import synth
from test_oracle_poly import kronecker_negacyclic

M32 = (1 << 32) - 1
MU = 1 << 29
TRUTH = {
    oracle.AND: lambda a, b: a & b, oracle.NAND: lambda a, b: 1 - (a & b),
    oracle.OR: lambda a, b: a | b, oracle.NOR: lambda a, b: 1 - (a | b),
    oracle.XOR: lambda a, b: a ^ b, oracle.XNOR: lambda a, b: 1 - (a ^ b),
    oracle.ANDNY: lambda a, b: (1 - a) & b, oracle.ANDYN: lambda a, b: a & (1 - b),
    oracle.ORNY: lambda a, b: (1 - a) | b, oracle.ORYN: lambda a, b: a | (1 - b),
}


def trlwe_phase(acc, K):
    return ((acc[1].astype(np.int64) - kronecker_negacyclic(acc[0], K).astype(np.int64)) & M32).astype(np.uint32)


def rotated_testv(phibar, N, mu=MU):
    """X^(-phibar) * mu * sum_j X^j, coefficient by coefficient."""
    out = np.zeros(N, dtype=np.uint32)
    for k in range(N):
        u = (k + phibar) % (2 * N)
        out[k] = mu if u < N else (-mu) & M32
    return out


def special_keys(P, seed, zero_s=False):
    """Noiseless keys whose BK masks are multiples of 2^(32 - l*bg_bits), so that
    every ACC coefficient stays exactly decomposable and blind rotation is exact."""
    km = synth.key_material(seed=seed, n=P.n, N=P.N, l=P.l, ks_t=P.ks_t, ks_base_bits=P.ks_base_bits,
                            noiseless=True)
    shift = 32 - P.l * P.bg_bits
    km = dataclasses.replace(km, bk_a=(km.bk_a >> np.uint32(shift)) << np.uint32(shift))
    if zero_s:
        km = dataclasses.replace(km, s=np.zeros_like(km.s))
    return oracle.keygen(P, km)


def phibar_of(lwe, s, N):
    n = len(s)
    ab = [oracle.modswitch(int(x), N) for x in lwe]
    return (ab[n] - sum(ab[i] * int(s[i]) for i in range(n))) % (2 * N)


@pytest.mark.parametrize("which", ["toy", "paper"])
def test_blind_rotate_exact_closed_form(which, toy_keys):
    P = toy_keys.P if which == "toy" else oracle.paper_params()
    keys = special_keys(P, seed=11)
    rng = np.random.default_rng(5)
    for t in range(3 if which == "toy" else 1):
        lwe = rng.integers(0, 1 << 32, P.n + 1, dtype=np.uint64).astype(np.uint32)
        acc = oracle.blind_rotate(keys, lwe)
        assert np.array_equal(trlwe_phase(acc, keys.K), rotated_testv(phibar_of(lwe, keys.s, P.N), P.N))


def test_blind_rotate_zero_key_closed_form(toy_keys):
    P = toy_keys.P
    keys = special_keys(P, seed=12, zero_s=True)
    km = synth.key_material(seed=13, n=P.n, N=P.N, l=P.l, noiseless=True)
    keys = oracle.keygen(P, dataclasses.replace(km, s=np.zeros_like(km.s)))  # general masks
    lwe = np.random.default_rng(6).integers(0, 1 << 32, P.n + 1, dtype=np.uint64).astype(np.uint32)
    acc = oracle.blind_rotate(keys, lwe)
    assert np.array_equal(trlwe_phase(acc, keys.K), rotated_testv(oracle.modswitch(int(lwe[-1]), P.N), P.N))


def test_schoolbook_and_karatsuba_rotations_agree(toy_keys):
    lwe = np.random.default_rng(7).integers(0, 1 << 32, toy_keys.P.n + 1, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(oracle.blind_rotate(toy_keys, lwe, karatsuba=True),
                          oracle.blind_rotate(toy_keys, lwe, karatsuba=False))


@pytest.mark.parametrize("N", [256, 1024])
def test_sample_extract_phase_invariant(N):
    rng = np.random.default_rng(N)
    K = rng.integers(0, 2, N).astype(np.uint32)
    for _ in range(4):
        acc = rng.integers(0, 1 << 32, (2, N), dtype=np.uint64).astype(np.uint32)
        big = oracle.sample_extract(acc)
        assert int(oracle.phase(K, big)[0]) == int(trlwe_phase(acc, K)[0])


def test_key_switch_closed_form(toy_keys):
    P = toy_keys.P
    km = synth.key_material(seed=14, n=P.n, N=P.N, l=P.l, noiseless=True)
    keys = oracle.keygen(P, km)
    rng = np.random.default_rng(8)
    for _ in range(20):
        big = rng.integers(0, 1 << 32, P.N + 1, dtype=np.uint64).astype(np.uint32)
        out = oracle.key_switch(keys, big)
        rounded = ((big[:P.N].astype(np.uint64) + (1 << 15)) & 0xFFFF0000) & M32
        want = (int(big[P.N]) - int((rounded * keys.K.astype(np.uint64)).sum())) & M32
        assert int(oracle.phase(keys.s, out)[0]) == want


def _truth_inputs(keys, g, seed):
    n = keys.P.n
    rows = [(a, b) for a in (0, 1) for b in (0, 1)]
    lm = synth.lwe_material(8, n, seed=seed)
    cts = oracle.encrypt_bits(keys.s, [v for r in rows for v in r], lm)
    return rows, cts.reshape(4, 2, n + 1)


def test_gate_truth_tables_paper(paper_keys):
    for g, f in TRUTH.items():
        rows, inp = _truth_inputs(paper_keys, g, seed=100 + g)
        out = oracle.gate_batch(paper_keys, g, inp)
        assert list(oracle.decrypt_bits(paper_keys.s, out)) == [f(a, b) for a, b in rows], oracle.GATE_NAMES[g]
    rows = [(c, a, b) for c in (0, 1) for a in (0, 1) for b in (0, 1)]
    lm = synth.lwe_material(24, 630, seed=200)
    cts = oracle.encrypt_bits(paper_keys.s, [v for r in rows for v in r], lm).reshape(8, 3, 631)
    out = oracle.gate_batch(paper_keys, oracle.MUX, cts)
    assert list(oracle.decrypt_bits(paper_keys.s, out)) == [a if c else b for c, a, b in rows]


def test_gate_truth_tables_toy_many_trials(toy_keys):
    n = toy_keys.P.n
    reps = 40
    for g, f in TRUTH.items():
        bits = synth.Stream(300 + g, 2, 0).bits(2 * 4 * reps).reshape(-1, 2)
        lm = synth.lwe_material(bits.size, n, seed=400 + g)
        cts = oracle.encrypt_bits(toy_keys.s, bits.reshape(-1), lm).reshape(-1, 2, n + 1)
        out = oracle.gate_batch(toy_keys, g, cts)
        want = np.array([f(int(a), int(b)) for a, b in bits])
        assert np.array_equal(oracle.decrypt_bits(toy_keys.s, out), want), oracle.GATE_NAMES[g]


def test_bootstrap_noise_within_tfhe_bound(paper_keys):
    """Output-noise variance of blind rotation and of key switching stays under
    tfhe-2's bounds: Var_BR <= n(k+1)lN(Bg/2)^2 sigma_BK^2 + n(1+kN) eps^2 with
    eps = 2^-(l*bg_bits+1), and Var_KS <= N t sigma_KS^2 + N 2^-2(tB+1)."""
    k = paper_keys
    P = k.P
    n, N, l = P.n, P.N, P.l
    var_br = n * 2 * l * N * (64.0 ** 2) * 2.0 ** -50 + n * (1 + N) * 2.0 ** -44
    var_ks = N * P.ks_t * 2.0 ** -30 + N * 2.0 ** -34
    rng = np.random.default_rng(9)
    lwes = rng.integers(0, 1 << 32, (4, n + 1), dtype=np.uint64).astype(np.uint32)
    with ThreadPoolExecutor(4) as ex:
        accs = list(ex.map(lambda x: oracle.blind_rotate(k, x), lwes))
    errs = []
    for lwe, acc in zip(lwes, accs):
        ph = trlwe_phase(acc, k.K)
        want = rotated_testv(phibar_of(lwe, k.s, N), N)
        errs.append(((ph.astype(np.int64) - want) & M32).astype(np.uint32).view(np.int32) / 2.0 ** 32)
    v_br = float(np.var(np.concatenate(errs)))
    assert var_br / 100 < v_br <= var_br, (v_br, var_br)

    ks_err = []
    for t in range(600):
        big = rng.integers(0, 1 << 32, N + 1, dtype=np.uint64).astype(np.uint32)
        out = oracle.key_switch(k, big)
        d = (int(oracle.phase(k.s, out)[0]) - int(oracle.phase(k.K, big)[0])) & M32
        ks_err.append((d - (1 << 32) if d >= (1 << 31) else d) / 2.0 ** 32)
    v_ks = float(np.var(ks_err))
    assert var_ks / 100 < v_ks <= var_ks * 1.15, (v_ks, var_ks)
    # total standard deviation vs the 1/16 decryption margin (Section 2.2)
    assert np.sqrt(var_br + var_ks) < (1 / 16) / 8
