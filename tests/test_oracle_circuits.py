"""Pins of the oracle's mode circuits.

Plaintext level: the paper's algorithms (HomCompLeOPT / HomCompL, HomEqOPT,
HomSum) modelled on bits, checked exhaustively against the predicates their
theorems state, and the plaintext-database rewrites checked against them.
Encrypted level: the oracle's circuits at a toy parameter set decrypt to the
predicates on all input pairs at small widths; a real-parameter IdM-8 run
decrypts correctly."""
import itertools
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2506_12761_gb300 import synth


def bits_of(v, l):
    return [(v >> i) & 1 for i in range(l)]


def signed(v, l):
    return v - (1 << l) if v >> (l - 1) else v


# ---------------- plaintext models of the paper's algorithms ----------------

def mux(c, a, b):
    return a if c else b


def paper_comp(x1, x2, strict):
    """Alg. HomCompLeOPT (strict=False) / HomCompL (strict=True) on bit lists."""
    l = len(x1)
    t0 = x1[l - 1] ^ x2[l - 1]
    t1 = 0 if strict else 1
    txnor = [1 - (x1[i] ^ x2[i]) for i in range(l - 1)]
    for i in range(l - 1):
        t1 = mux(txnor[i], t1, x2[i])
    return mux(t0, x1[l - 1], t1)


def gate_fn(name):
    return {"AND": lambda a, b: a & b, "OR": lambda a, b: a | b,
            "ANDNY": lambda a, b: (1 - a) & b, "ORNY": lambda a, b: (1 - a) | b}[name]


def rewrite_comp(plain, x, l, plain_first, strict, unsigned):
    """The single-gate rewrite the oracle and the CUDA scheduler execute."""
    xb = bits_of(x, l)
    if unsigned:
        plain ^= 1 << (l - 1)
        xb[l - 1] ^= 1
    t = 0 if strict else 1
    for i in range(l - 1):
        b = (plain >> i) & 1
        g = ("AND" if b else "OR") if plain_first else ("ORNY" if b else "ANDNY")
        t = gate_fn(g)(xb[i], t)
    tb = (plain >> (l - 1)) & 1
    g = ("ORNY" if tb else "ANDNY") if plain_first else ("AND" if tb else "OR")
    return gate_fn(g)(xb[l - 1], t)


def paper_eq_tree(x1, x2):
    """Alg. HomEqOPT on bit lists."""
    l = len(x1)
    t = [1 - (x1[i] ^ x2[i]) for i in range(l)]
    k = 1
    while k < l:
        for i in range(0, l, 2 * k):
            if i + k < l:
                t[i] = t[i] & t[i + k]
        k *= 2
    return t[0]


@pytest.mark.parametrize("l", [2, 3, 4, 5, 6])
def test_paper_comparators_are_signed_le_lt(l):
    for z1, z2 in itertools.product(range(1 << l), repeat=2):
        b1, b2 = bits_of(z1, l), bits_of(z2, l)
        assert paper_comp(b1, b2, False) == int(signed(z1, l) <= signed(z2, l))
        assert paper_comp(b1, b2, True) == int(signed(z1, l) < signed(z2, l))


@pytest.mark.parametrize("l", [2, 3, 4, 5, 6, 7])
def test_plaintext_rewrites_equal_paper_algorithm(l):
    for a, x in itertools.product(range(1 << l), repeat=2):
        # HomCompLE(a, x) with a plaintext, and HomCompL(x, b) with b = a plaintext
        assert rewrite_comp(a, x, l, True, False, False) == paper_comp(bits_of(a, l), bits_of(x, l), False)
        assert rewrite_comp(a, x, l, False, True, False) == paper_comp(bits_of(x, l), bits_of(a, l), True)
        # unsigned variant through the top-bit flip
        assert rewrite_comp(a, x, l, True, False, True) == int(a <= x)
        assert rewrite_comp(a, x, l, False, True, True) == int(x < a)


@pytest.mark.parametrize("l", [1, 2, 3, 5, 6, 8])
def test_paper_eq_tree_is_equality(l):
    for z1, z2 in itertools.product(range(1 << l), repeat=2):
        assert paper_eq_tree(bits_of(z1, l), bits_of(z2, l)) == int(z1 == z2)


@pytest.mark.parametrize("M", list(range(1, 18)) + [64, 100])
def test_homsum_tree_selects_the_one_hot_entry(M):
    rng = np.random.default_rng(M)
    vals = [0] * M
    kappa = int(rng.integers(0, M))
    vals[kappa] = int(rng.integers(0, 1 << 16))
    S = list(vals)
    k = 1
    xors = 0
    while k < M:
        for i in range(0, M, 2 * k):
            if i + k < M:
                S[i] ^= S[i + k]
                xors += 1
        k *= 2
    assert S[0] == vals[kappa] and xors == M - 1


def test_gate_counts_per_entry():
    """131 bootstraps per IntV entry, 31 per CoV-16+16 entry, l-1 per IdM-l entry."""
    assert 4 * 32 + 3 == 131 and 2 * 15 + 1 == 31
    assert 1024 * 131 == 134144 and 65536 * 31 == 2031616 and 32 * (65536 - 1) == 2097120


# ---------------- encrypted circuits at toy parameters ----------------

def enc_value(keys, v, l, seed):
    lm = synth.lwe_material(l, keys.P.n, seed=seed)
    return oracle.encrypt_bits(keys.s, bits_of(v, l), lm)


def pmap(f, items):
    with ThreadPoolExecutor(8) as ex:
        return list(ex.map(f, items))


def test_toy_plain_comparators_all_pairs(toy_keys):
    l = 4
    xs = {x: enc_value(toy_keys, x, l, 1000 + x) for x in range(1 << l)}
    jobs = list(itertools.product(range(1 << l), range(1 << l), [False, True]))

    def run(job):
        a, x, uns = job
        le = oracle.comp_plain(toy_keys, xs[x], a, True, False, uns)
        lt = oracle.comp_plain(toy_keys, xs[x], a, False, True, uns)
        return oracle.decrypt_bits(toy_keys.s, np.stack([le, lt]))

    for (a, x, uns), got in zip(jobs, pmap(run, jobs)):
        if uns:
            want = [int(a <= x), int(x < a)]
        else:
            want = [int(signed(a, l) <= signed(x, l)), int(signed(x, l) < signed(a, l))]
        assert list(got) == want, (a, x, uns)


def test_toy_encrypted_paper_comparators(toy_keys):
    l = 3
    cts = {v: enc_value(toy_keys, v, l, 2000 + v) for v in range(1 << l)}
    jobs = list(itertools.product(range(1 << l), repeat=2))

    def run(job):
        z1, z2 = job
        return oracle.decrypt_bits(toy_keys.s, np.stack([oracle.comp_enc(toy_keys, cts[z1], cts[z2], False),
                                                         oracle.comp_enc(toy_keys, cts[z1], cts[z2], True)]))

    for (z1, z2), got in zip(jobs, pmap(run, jobs)):
        assert list(got) == [int(signed(z1, l) <= signed(z2, l)), int(signed(z1, l) < signed(z2, l))]


def test_toy_equality_all_pairs(toy_keys):
    l = 4
    xs = {x: enc_value(toy_keys, x, l, 3000 + x) for x in range(1 << l)}
    jobs = list(itertools.product(range(1 << l), repeat=2))
    got = pmap(lambda j: oracle.decrypt_bits(toy_keys.s, oracle.eq_plain(toy_keys, xs[j[0]], j[1]))[0], jobs)
    assert [int(g) for g in got] == [int(x == v) for x, v in jobs]
    jobs3 = list(itertools.product(range(8), repeat=2))
    got = pmap(lambda j: oracle.decrypt_bits(toy_keys.s, oracle.eq_enc(
        toy_keys, enc_value(toy_keys, j[0], 3, 4000 + j[0]), enc_value(toy_keys, j[1], 3, 4100 + j[1])))[0], jobs3)
    assert [int(g) for g in got] == [int(a == b) for a, b in jobs3]


def test_toy_intv_cov_idm(toy_keys):
    l = 8
    st = synth.Stream(77, 3, 0)
    x, y = (int(v) for v in st.words(2) & np.uint32(0xFF))
    cx, cy = enc_value(toy_keys, x, l, 5000), enc_value(toy_keys, y, l, 5001)
    rects = []
    for d in range(24):
        r = []
        for ax, q in ((0, x), (1, y)):
            if d % 3 == 0:   # make some rectangles contain the point
                lo, hi = max(0, q - int(st.words(1)[0] % 5)), min(255, q + 1 + int(st.words(1)[0] % 5))
            else:
                u, v = sorted(int(w) & 0xFF for w in st.words(2))
                lo, hi = u, v if v > u else u + 1
            r += [lo, hi]
        rects.append(r)
    out = oracle.intv_batch(toy_keys, cx, cy, rects, unsigned=True)
    want = [int(r[0] <= x < r[1] and r[2] <= y < r[3]) for r in rects]
    assert list(oracle.decrypt_bits(toy_keys.s, out)) == want and sum(want) > 0

    w = 4
    cell = (5 << w) | 9
    ccts = enc_value(toy_keys, cell, 2 * w, 6000)
    cells = [cell, (5 << w) | 8, (4 << w) | 9, cell, 0, 255]
    out = oracle.cov_batch(toy_keys, ccts, cells, width=w)
    assert list(oracle.decrypt_bits(toy_keys.s, out)) == [int(c == cell) for c in cells]

    ids = [3, 17, 40, 17, 63, 0, 1, 2, 9]
    q = 40
    xq = enc_value(toy_keys, q, 6, 7000)
    out = oracle.idm_batch(toy_keys, xq, ids)
    assert list(oracle.decrypt_bits(toy_keys.s, out)) == [int(i == q) for i in ids]
    payload = [11, 22, 29, 4, 7, 1, 0, 31, 16]
    agg = oracle.idm_payload(toy_keys, xq, ids, payload, payload_bits=5)
    assert list(oracle.decrypt_bits(toy_keys.s, agg)) == bits_of(payload[ids.index(q)], 5)


def test_paper_params_idm8_d4(paper_keys):
    """The smallest workload at the paper's parameters: 8-bit id, D = 4."""
    w = synth.idm_workload(4, 8)
    x = enc_value(paper_keys, w["query"], 8, 8000)
    out = oracle.idm_batch(paper_keys, x, w["ids"])
    assert list(oracle.decrypt_bits(paper_keys.s, out)) == [int(i == w["query"]) for i in w["ids"]]
