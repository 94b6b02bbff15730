"""ctypes wrapper over tfhe_oracle.c (test infrastructure only; see tfhe_oracle.c)."""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tfhe_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

AND, NAND, OR, NOR, XOR, XNOR, ANDNY, ANDYN, ORNY, ORYN, MUX = range(11)
GATE_NAMES = ["AND", "NAND", "OR", "NOR", "XOR", "XNOR", "ANDNY", "ANDYN", "ORNY", "ORYN", "MUX"]
MU = 1 << 29  # 1/8 on the 32-bit torus


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("N", ctypes.c_int32), ("l", ctypes.c_int32),
                ("bg_bits", ctypes.c_int32), ("ks_t", ctypes.c_int32), ("ks_base_bits", ctypes.c_int32)]

    @property
    def base(self):
        return 1 << self.ks_base_bits


def paper_params() -> Params:
    """TFHE 128-bit set used by the paper (Appendix, TFHE parameter table)."""
    return Params(630, 1024, 3, 7, 8, 2)


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host C compiler (no GPU involved)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-Wall", "-Wno-unused-function", SRC, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.POINTER(Params)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i = ctypes.c_int
        i64 = ctypes.c_int64
        u32 = ctypes.c_uint32
        sig = {
            "orc_poly_mul_schoolbook": (None, [u32p, u32p, u32p, i]),
            "orc_poly_mul_karatsuba": (None, [u32p, u32p, u32p, i]),
            "orc_poly_mul_xe": (None, [u32p, u32p, i, i]),
            "orc_lwe_phase": (u32, [i, u32p, u32p]),
            "orc_lwe_encrypt": (None, [i, u32p, u32p, u32, u32, u32p]),
            "orc_lwe_decrypt_bit": (i, [i, u32p, u32p]),
            "orc_keygen_bk": (None, [P, u32p, u32p, u32p, u32p, u32p]),
            "orc_keygen_ksk": (None, [P, u32p, u32p, u32p, u32p, u32p]),
            "orc_modswitch": (u32, [u32, i]),
            "orc_decompose": (None, [P, u32, i32p]),
            "orc_blind_rotate": (None, [P, u32p, u32p, u32, u32p, i]),
            "orc_sample_extract": (None, [i, u32p, u32p]),
            "orc_key_switch": (None, [P, u32p, u32p, u32p]),
            "orc_bootstrap": (None, [P, u32p, u32p, u32p, u32p]),
            "orc_gate_combine": (None, [i, i, u32p, u32p, u32p]),
            "orc_gate": (None, [P, u32p, u32p, i, u32p, u32p, u32p, u32p]),
            "orc_gate_batch": (None, [P, u32p, u32p, i, u32p, u32p, i64, i]),
            "orc_eq_plain": (None, [P, u32p, u32p, u32p, i, ctypes.c_uint64, u32p]),
            "orc_eq_enc": (None, [P, u32p, u32p, u32p, u32p, i, u32p]),
            "orc_comp_enc": (None, [P, u32p, u32p, u32p, u32p, i, i, u32p]),
            "orc_comp_plain": (None, [P, u32p, u32p, u32p, ctypes.c_uint64, i, i, i, i, u32p]),
            "orc_intv_entry": (None, [P, u32p, u32p, u32p, u32p, i, u64p, i, u32p]),
            "orc_cov_entry": (None, [P, u32p, u32p, u32p, i, ctypes.c_uint64, ctypes.c_uint64, u32p]),
            "orc_idm_batch": (None, [P, u32p, u32p, u32p, i, u64p, i64, u32p, i]),
            "orc_intv_batch": (None, [P, u32p, u32p, u32p, u32p, i, u64p, i64, i, u32p, i]),
            "orc_cov_batch": (None, [P, u32p, u32p, u32p, i, u64p, i64, u32p, i]),
            "orc_zero_out_plain": (None, [i, u32p, i, u32p]),
            "orc_homsum_tree": (None, [P, u32p, u32p, u32p, i64, i, i]),
            "orc_gate_linear": (None, [P, u32p, u32p, i, i, i32p, u32p, u32p, u32, u32p]),
            "orc_gate_linear_batch": (None, [P, u32p, u32p, i64, i32p, i32p, i32p, u32p, u32p, u32p, u32p, i]),
            "orc_xor_many": (None, [P, u32p, u32p, u32p, i, u32p]),
            "orc_homsum_tree_fanin": (None, [P, u32p, u32p, u32p, i64, i, i, i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray, ct=ctypes.c_uint32):
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be C-contiguous"
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def default_threads() -> int:
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


# --------------------------------------------------------------------------
# Polynomials
# --------------------------------------------------------------------------

def poly_mul_schoolbook(a, b):
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    lib().orc_poly_mul_schoolbook(_p(out), _p(a), _p(b), len(a))
    return out


def poly_mul_karatsuba(a, b):
    a, b = _u32(a), _u32(b)
    out = np.zeros_like(a)
    lib().orc_poly_mul_karatsuba(_p(out), _p(a), _p(b), len(a))
    return out


def poly_mul_xe(p, e: int):
    p = _u32(p)
    out = np.zeros_like(p)
    lib().orc_poly_mul_xe(_p(out), _p(p), int(e), len(p))
    return out


# --------------------------------------------------------------------------
# Keys
# --------------------------------------------------------------------------

@dataclass
class Keys:
    P: Params
    s: np.ndarray     # [n]
    K: np.ndarray     # [N]
    bk: np.ndarray    # [n][2l][2][N]
    ksk: np.ndarray   # [N][t][base][n+1]


def keygen(P: Params, km) -> Keys:
    """Cloud key from synth.KeyMaterial (BK = TRGSW encryptions of s_i, KSK)."""
    s, K = _u32(km.s), _u32(km.K)
    bk_a, bk_e, ksk_a, ksk_e = _u32(km.bk_a), _u32(km.bk_e), _u32(km.ksk_a), _u32(km.ksk_e)
    bk = np.zeros((P.n, 2 * P.l, 2, P.N), dtype=np.uint32)
    ksk = np.zeros((P.N, P.ks_t, P.base, P.n + 1), dtype=np.uint32)
    lib().orc_keygen_bk(ctypes.byref(P), _p(s), _p(K), _p(bk_a), _p(bk_e), _p(bk))
    lib().orc_keygen_ksk(ctypes.byref(P), _p(s), _p(K), _p(ksk_a), _p(ksk_e), _p(ksk))
    return Keys(P, s, K, bk, ksk)


# --------------------------------------------------------------------------
# LWE
# --------------------------------------------------------------------------

def encrypt_mu(s, a, e, mu) -> np.ndarray:
    """LWE encryptions of torus values mu[i] with masks a[i] and noises e[i]."""
    s = _u32(s)
    a = _u32(a).reshape(-1, len(s))
    e = _u32(e).reshape(-1)
    mu = _u32(mu).reshape(-1)
    n = len(s)
    out = np.zeros((a.shape[0], n + 1), dtype=np.uint32)
    for i in range(a.shape[0]):
        lib().orc_lwe_encrypt(n, _p(s), _p(a[i]), int(e[i]), int(mu[i]), _p(out[i]))
    return out


def encrypt_bits(s, bits, lwe_mat) -> np.ndarray:
    bits = np.asarray(bits).reshape(-1)
    mu = np.where(bits != 0, MU, (1 << 32) - MU).astype(np.uint32)
    return encrypt_mu(s, lwe_mat.a[: len(bits)], lwe_mat.e[: len(bits)], mu)


def server_encrypt(pk, bits) -> np.ndarray:
    """Alg. ServerEnc: ct = (0, Ecd(bit)) + pk for one public-key ciphertext
    pk (an encryption of zero from Alg. PubKeyGen, i.e. encrypt_mu with mu = 0)
    per bit; Ecd(1) = 1/8, Ecd(0) = -1/8 (Section 2.2)."""
    pk = _u32(pk).reshape(-1, _u32(pk).shape[-1]).copy()
    bits = np.asarray(bits).reshape(-1)
    pk[:, -1] += np.where(bits != 0, MU, (1 << 32) - MU).astype(np.uint32)
    return pk


def phase(s, ct) -> np.ndarray:
    s = _u32(s)
    ct = _u32(ct).reshape(-1, len(s) + 1)
    return np.array([lib().orc_lwe_phase(len(s), _p(s), _p(ct[i])) for i in range(ct.shape[0])],
                    dtype=np.uint32)


def decrypt_bits(s, ct) -> np.ndarray:
    return (phase(s, ct).view(np.int32) >= 0).astype(np.uint32)


def trivial(n: int, mu: int) -> np.ndarray:
    c = np.zeros(n + 1, dtype=np.uint32)
    c[n] = mu & 0xFFFFFFFF
    return c


def lwe_not(c) -> np.ndarray:
    return (np.uint32(0) - _u32(c)).astype(np.uint32)


# --------------------------------------------------------------------------
# Bootstrapping stages
# --------------------------------------------------------------------------

def modswitch(x: int, N: int) -> int:
    return int(lib().orc_modswitch(int(x) & 0xFFFFFFFF, N))


def decompose(P: Params, x: int) -> np.ndarray:
    d = np.zeros(16, dtype=np.int32)
    lib().orc_decompose(ctypes.byref(P), int(x) & 0xFFFFFFFF, _p(d, ctypes.c_int32))
    return d[: P.l].copy()


def blind_rotate(keys: Keys, lwe, mu: int = MU, karatsuba: bool = True) -> np.ndarray:
    P = keys.P
    lwe = _u32(lwe)
    acc = np.zeros((2, P.N), dtype=np.uint32)
    lib().orc_blind_rotate(ctypes.byref(P), _p(keys.bk), _p(lwe), mu & 0xFFFFFFFF, _p(acc), int(karatsuba))
    return acc


def sample_extract(acc) -> np.ndarray:
    acc = _u32(acc)
    N = acc.shape[-1]
    big = np.zeros(N + 1, dtype=np.uint32)
    lib().orc_sample_extract(N, _p(acc), _p(big))
    return big


def key_switch(keys: Keys, big) -> np.ndarray:
    P = keys.P
    big = _u32(big)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_key_switch(ctypes.byref(P), _p(keys.ksk), _p(big), _p(out))
    return out


def bootstrap(keys: Keys, lwe) -> np.ndarray:
    P = keys.P
    lwe = _u32(lwe)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_bootstrap(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(lwe), _p(out))
    return out


def gate_combine(gate: int, c1, c2) -> np.ndarray:
    c1, c2 = _u32(c1), _u32(c2)
    out = np.zeros_like(c1)
    lib().orc_gate_combine(len(c1) - 1, gate, _p(c1), _p(c2), _p(out))
    return out


def gate(keys: Keys, g: int, c1, c2, c3=None) -> np.ndarray:
    P = keys.P
    c1, c2 = _u32(c1), _u32(c2)
    c3 = _u32(c3) if c3 is not None else np.zeros(P.n + 1, dtype=np.uint32)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_gate(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), g, _p(c1), _p(c2), _p(c3), _p(out))
    return out


def gate_batch(keys: Keys, g: int, inputs, threads: int | None = None) -> np.ndarray:
    """inputs: [count][arity][n+1] (arity 3 for MUX)."""
    P = keys.P
    inputs = _u32(inputs)
    count = inputs.shape[0]
    out = np.zeros((count, P.n + 1), dtype=np.uint32)
    if count:
        lib().orc_gate_batch(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), g, _p(inputs), _p(out),
                             count, threads or default_threads())
    return out


# --------------------------------------------------------------------------
# Circuits
# --------------------------------------------------------------------------

def eq_plain(keys: Keys, x_cts, value: int) -> np.ndarray:
    P = keys.P
    x = _u32(x_cts)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_eq_plain(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(x), x.shape[0], int(value), _p(out))
    return out


def eq_enc(keys: Keys, x_cts, y_cts) -> np.ndarray:
    P = keys.P
    x, y = _u32(x_cts), _u32(y_cts)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_eq_enc(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(x), _p(y), x.shape[0], _p(out))
    return out


def comp_enc(keys: Keys, c1, c2, strict: bool) -> np.ndarray:
    P = keys.P
    c1, c2 = _u32(c1), _u32(c2)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_comp_enc(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(c1), _p(c2), c1.shape[0],
                       int(strict), _p(out))
    return out


def comp_plain(keys: Keys, x_cts, plain: int, plain_first: bool, strict: bool, unsigned: bool) -> np.ndarray:
    P = keys.P
    x = _u32(x_cts)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_comp_plain(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(x), int(plain), x.shape[0],
                         int(plain_first), int(strict), int(unsigned), _p(out))
    return out


def intv_batch(keys: Keys, cx, cy, rects, unsigned: bool = True, threads: int | None = None) -> np.ndarray:
    P = keys.P
    cx, cy = _u32(cx), _u32(cy)
    rects = np.ascontiguousarray(np.asarray(rects, dtype=np.uint64).reshape(-1, 4))
    D = rects.shape[0]
    out = np.zeros((D, P.n + 1), dtype=np.uint32)
    if D:
        lib().orc_intv_batch(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(cx), _p(cy), cx.shape[0],
                             _p(rects, ctypes.c_uint64), D, int(unsigned), _p(out), threads or default_threads())
    return out


def idm_batch(keys: Keys, x_cts, ids, threads: int | None = None) -> np.ndarray:
    P = keys.P
    x = _u32(x_cts)
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64).reshape(-1))
    D = ids.shape[0]
    out = np.zeros((D, P.n + 1), dtype=np.uint32)
    if D:
        lib().orc_idm_batch(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(x), x.shape[0],
                            _p(ids, ctypes.c_uint64), D, _p(out), threads or default_threads())
    return out


def cov_batch(keys: Keys, cell_cts, cells, width: int = 16, threads: int | None = None) -> np.ndarray:
    """cells: packed (y << width) | x plaintext cells."""
    P = keys.P
    c = _u32(cell_cts)
    cells = np.asarray(cells, dtype=np.uint64).reshape(-1)
    locs = np.ascontiguousarray(np.stack([cells & ((1 << width) - 1), cells >> width], axis=1).astype(np.uint64))
    D = cells.shape[0]
    out = np.zeros((D, P.n + 1), dtype=np.uint32)
    if D:
        lib().orc_cov_batch(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(c), width,
                            _p(locs, ctypes.c_uint64), D, _p(out), threads or default_threads())
    return out


def zero_out_plain(v, bit: int) -> np.ndarray:
    v = _u32(v)
    out = np.zeros_like(v)
    lib().orc_zero_out_plain(len(v) - 1, _p(v), int(bit), _p(out))
    return out


def homsum_tree(keys: Keys, S, threads: int | None = None) -> np.ndarray:
    """S: [M][lS][n+1]; returns the aggregated [lS][n+1] (pairwise XOR tree)."""
    P = keys.P
    S = _u32(S).copy()
    M, lS = S.shape[0], S.shape[1]
    if M:
        lib().orc_homsum_tree(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(S), M, lS,
                              threads or default_threads())
    return S[0].copy()


def homsum_tree_fanin(keys: Keys, S, g: int, threads: int | None = None) -> np.ndarray:
    """S: [M][lS][n+1]; the fan-in-g XOR tree (one bootstrap per g inputs).
    Returns the aggregated [lS][n+1]; g = 2 is homsum_tree."""
    P = keys.P
    S = _u32(S).copy()
    M, lS = S.shape[0], S.shape[1]
    if M:
        lib().orc_homsum_tree_fanin(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(S), M, lS, int(g),
                                    threads or default_threads())
    return S[0].copy()


def xor_many(keys: Keys, cts) -> np.ndarray:
    """XOR of g ciphertexts [g][n+1] with one bootstrap of 2 sum c_k + T((g-1)/4)."""
    P = keys.P
    c = _u32(cts)
    out = np.zeros(P.n + 1, dtype=np.uint32)
    lib().orc_xor_many(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), _p(c), c.shape[0], _p(out))
    return out


def gate_linear_batch(keys: Keys, nrot, nin, coef, cst, ks_cst, inputs, threads: int | None = None) -> np.ndarray:
    """Gates given by their pre-combinations: rotation r of gate g blind-rotates
    sum_k coef[g][r][k] inputs[g][k] + T(cst[g][r]); the extractions are summed
    with T(ks_cst[g]) and key-switched.  nrot, nin, ks_cst: [count];
    coef: [count][2][8]; cst: [count][2]; inputs: [count][8][n+1]."""
    P = keys.P
    i32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    nrot, nin, coef = i32(nrot), i32(nin), i32(coef)
    cst, ks_cst, inputs = _u32(cst), _u32(ks_cst), _u32(inputs)
    count = nrot.shape[0]
    assert coef.shape == (count, 2, 8) and cst.shape == (count, 2) and inputs.shape == (count, 8, P.n + 1)
    out = np.zeros((count, P.n + 1), dtype=np.uint32)
    if count:
        lib().orc_gate_linear_batch(ctypes.byref(P), _p(keys.bk), _p(keys.ksk), count, _p(nrot, ctypes.c_int32),
                                    _p(nin, ctypes.c_int32), _p(coef, ctypes.c_int32), _p(cst), _p(ks_cst),
                                    _p(inputs), _p(out), threads or default_threads())
    return out


def idm_payload(keys: Keys, x_cts, ids, payload, payload_bits: int = 32, threads: int | None = None,
                fanin: int = 2) -> np.ndarray:
    """IdM with a plaintext payload per entry: match bits, free zero-out with
    each payload bit, then the HomSum XOR tree (pairwise, or fan-in g with one
    bootstrap per g inputs).  Returns [payload_bits][n+1]."""
    P = keys.P
    v = idm_batch(keys, x_cts, ids, threads)
    pay = np.asarray(payload, dtype=np.uint64).reshape(-1)
    D = len(pay)
    S = np.zeros((D, payload_bits, P.n + 1), dtype=np.uint32)
    for d in range(D):
        for j in range(payload_bits):
            S[d, j] = zero_out_plain(v[d], int((int(pay[d]) >> j) & 1))
    if fanin == 2:
        return homsum_tree(keys, S, threads)
    return homsum_tree_fanin(keys, S, fanin, threads)


# --------------------------------------------------------------------------
# Encrypted database (Section 3.2: the database bits are ServerEnc ciphertexts)
# --------------------------------------------------------------------------

def _pool(threads):
    return ThreadPoolExecutor(max_workers=threads or default_threads())


def comp_enc_unsigned(keys: Keys, c1, c2, strict: bool) -> np.ndarray:
    """c1 <= c2 (strict: c1 < c2) as unsigned l-bit integers: Alg.
    HomCompLeOPT / HomCompL (comp_enc, signed two's complement) on operands
    whose top bits are both negated."""
    c1, c2 = _u32(c1).copy(), _u32(c2).copy()
    c1[-1] = lwe_not(c1[-1])
    c2[-1] = lwe_not(c2[-1])
    return comp_enc(keys, c1, c2, strict)


def intv_enc_batch(keys: Keys, cx, cy, enc_rects, threads: int | None = None) -> np.ndarray:
    """Alg. InterValid with encrypted bounds: AND(AND(LE(x_lo,x), L(x,x_hi)),
    AND(LE(y_lo,y), L(y,y_hi))).  enc_rects: [D][4][l][n+1] (x_lo, x_hi, y_lo,
    y_hi).  The four comparators of all entries run on a thread pool."""
    cx, cy = _u32(cx), _u32(cy)
    R = _u32(enc_rects)
    D = R.shape[0]
    jobs = []
    for d in range(D):
        jobs += [(R[d, 0], cx, False), (cx, R[d, 1], True), (R[d, 2], cy, False), (cy, R[d, 3], True)]
    with _pool(threads) as ex:
        v = list(ex.map(lambda j: comp_enc_unsigned(keys, *j), jobs))
        vx = list(ex.map(lambda d: gate(keys, AND, v[4 * d], v[4 * d + 1]), range(D)))
        vy = list(ex.map(lambda d: gate(keys, AND, v[4 * d + 2], v[4 * d + 3]), range(D)))
        out = list(ex.map(lambda d: gate(keys, AND, vx[d], vy[d]), range(D)))
    return np.stack(out) if D else np.zeros((0, keys.P.n + 1), np.uint32)


def cov_enc_batch(keys: Keys, cell_cts, enc_cells, width: int, threads: int | None = None) -> np.ndarray:
    """Alg. CoV with encrypted cells: AND(HomEqOPT(x, loc_x), HomEqOPT(y, loc_y)),
    both equality tests with bootstrapped XNORs (eq_enc).  cell_cts: [2w][n+1]
    (x bits then y bits); enc_cells: [D][2w][n+1]."""
    c = _u32(cell_cts)
    E = _u32(enc_cells)
    D = E.shape[0]
    with _pool(threads) as ex:
        vx = list(ex.map(lambda d: eq_enc(keys, c[:width], E[d, :width]), range(D)))
        vy = list(ex.map(lambda d: eq_enc(keys, c[width:], E[d, width:]), range(D)))
        out = list(ex.map(lambda d: gate(keys, AND, vx[d], vy[d]), range(D)))
    return np.stack(out) if D else np.zeros((0, keys.P.n + 1), np.uint32)


def idm_enc_batch(keys: Keys, x_cts, enc_ids, threads: int | None = None) -> np.ndarray:
    """IdM match bits with encrypted ids (eq_enc per entry).  enc_ids: [D][l][n+1]."""
    x = _u32(x_cts)
    E = _u32(enc_ids)
    with _pool(threads) as ex:
        out = list(ex.map(lambda d: eq_enc(keys, x, E[d]), range(E.shape[0])))
    return np.stack(out) if out else np.zeros((0, keys.P.n + 1), np.uint32)


def aggregate_enc(keys: Keys, v, enc_payload, threads: int | None = None, fanin: int = 2) -> np.ndarray:
    """Alg. HomBitwiseAND with encrypted payloads (one bootstrapped AND of each
    entry's validation bit v[d] with each of its payload bits), then the
    HomSum XOR tree (fanin 2) or the fan-in-g tree of homsum_tree_fanin.
    enc_payload: [D][lS][n+1]; returns [lS][n+1]."""
    v = _u32(v)
    Pay = _u32(enc_payload)
    D, lS = Pay.shape[0], Pay.shape[1]
    with _pool(threads) as ex:
        flat = list(ex.map(lambda k: gate(keys, AND, v[k // lS], Pay[k // lS, k % lS]), range(D * lS)))
    S = np.stack(flat).reshape(D, lS, -1)
    if fanin > 2:
        return homsum_tree_fanin(keys, S, fanin, threads)
    return homsum_tree(keys, S, threads)


def idm_enc_payload(keys: Keys, x_cts, enc_ids, enc_payload, threads: int | None = None) -> np.ndarray:
    """IdM with an encrypted payload: match bits (idm_enc_batch), then
    aggregate_enc.  Returns [lS][n+1]."""
    return aggregate_enc(keys, idm_enc_batch(keys, x_cts, enc_ids, threads), enc_payload, threads)
