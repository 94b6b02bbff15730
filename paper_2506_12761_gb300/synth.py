"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle tests.

This module draws random numbers and nothing else: it holds none of TFHE's
arithmetic (no encryption, no key generation, no polynomial products).  Every
random quantity the method consumes -- key bits, uniform mask words, Gaussian
noise integers, plaintext databases, query values, arrival times -- is produced
here and handed to whichever side (the CUDA library's client or the oracle)
combines it.

Generator: ChaCha20 block function as defined in RFC 8439 section 2.3
(20 rounds, 32-bit little-endian words).  A stream is addressed by
(seed, stream id, substream id):
    key   = [seed_lo, seed_hi, stream, substream, 0, 0, 0, 0]
    nonce = [0, 0, 0], block counter 0, 1, 2, ...
The word sequence is the concatenation of the blocks' 16 output words.

Derived draws:
  * uniform torus word  = the next 32-bit word (T = R/Z with 1.0 == 2^32).
  * Gaussian noise       = Box-Muller on two 53-bit uniforms in float64,
                          e = rint(sigma * 2^32 * z) reduced mod 2^32.  The
                          paper (Section 2.2, TLWE definition) only says the
                          error is Gaussian; this discretisation is our reading.
  * key bit              = word & 1 (binary keys, Section 2.2 TLWE definition).

Stream ids (master seed 20250615): 1 keys, 2 query encryption, 3 database,
4 arrivals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 20250615
STREAM_KEYS = 1
STREAM_QUERY = 2
STREAM_DB = 3
STREAM_ARRIVALS = 4
STREAM_PUBKEY = 5   # Alg. PubKeyGen material (masks and noises of the encryptions of zero)

_SIGMA = np.uint32(0x61707865), np.uint32(0x3320646E), np.uint32(0x79622D32), np.uint32(0x6B206574)

# The paper's 128-bit parameter set (Appendix, TFHE parameter table).
PAPER_PARAMS = dict(n=630, N=1024, k=1, l=3, bg_bits=7, ks_t=8, ks_base_bits=2)
SIGMA_LWE_LOG2 = -15   # fresh LWE encryptions and KSK rows (sigma_KS = 2^-15)
SIGMA_KS_LOG2 = -15
SIGMA_BK_LOG2 = -25


def _rotl(x, r):
    return (x << np.uint32(r)) | (x >> np.uint32(32 - r))


def _quarter(s, a, b, c, d):
    s[a] += s[b]; s[d] ^= s[a]; s[d] = _rotl(s[d], 16)
    s[c] += s[d]; s[b] ^= s[c]; s[b] = _rotl(s[b], 12)
    s[a] += s[b]; s[d] ^= s[a]; s[d] = _rotl(s[d], 8)
    s[c] += s[d]; s[b] ^= s[c]; s[b] = _rotl(s[b], 7)


def chacha20_blocks(key8, nonce3, counter0: int, nblocks: int) -> np.ndarray:
    """RFC 8439 ChaCha20 block function applied to counters counter0..counter0+nblocks-1.

    Returns a (nblocks, 16) uint32 array of output words (the serialised
    keystream block is these words in little-endian byte order)."""
    key8 = [np.uint32(k) for k in key8]
    nonce3 = [np.uint32(v) for v in nonce3]
    ctr = (np.arange(nblocks, dtype=np.uint64) + np.uint64(counter0)).astype(np.uint32)
    init = [np.full(nblocks, w, dtype=np.uint32) for w in (*_SIGMA, *key8)]
    init.append(ctr)
    init += [np.full(nblocks, w, dtype=np.uint32) for w in nonce3]
    s = [x.copy() for x in init]
    with np.errstate(over="ignore"):
        for _ in range(10):
            _quarter(s, 0, 4, 8, 12); _quarter(s, 1, 5, 9, 13)
            _quarter(s, 2, 6, 10, 14); _quarter(s, 3, 7, 11, 15)
            _quarter(s, 0, 5, 10, 15); _quarter(s, 1, 6, 11, 12)
            _quarter(s, 2, 7, 8, 13); _quarter(s, 3, 4, 9, 14)
        out = np.stack([s[i] + init[i] for i in range(16)], axis=1)
    return out


class Stream:
    """A sequential reader over one (seed, stream, substream) ChaCha20 keystream."""

    def __init__(self, seed: int = MASTER_SEED, stream: int = STREAM_KEYS, substream: int = 0):
        self.key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, stream & 0xFFFFFFFF,
                    substream & 0xFFFFFFFF, 0, 0, 0, 0]
        self.pos = 0  # words consumed

    def words(self, count: int) -> np.ndarray:
        count = int(count)
        if count == 0:
            return np.zeros(0, dtype=np.uint32)
        b0 = self.pos // 16
        b1 = (self.pos + count + 15) // 16
        blk = chacha20_blocks(self.key, (0, 0, 0), b0, b1 - b0).reshape(-1)
        off = self.pos - b0 * 16
        self.pos += count
        return blk[off:off + count].copy()

    def torus(self, shape) -> np.ndarray:
        shape = tuple(np.atleast_1d(shape)) if not isinstance(shape, tuple) else shape
        return self.words(int(np.prod(shape))).reshape(shape)

    def bits(self, shape) -> np.ndarray:
        return (self.torus(shape) & np.uint32(1)).astype(np.uint32)

    def unit_doubles(self, count: int) -> np.ndarray:
        """`count` float64 values in [0, 1) with 53 random bits each (two words per value)."""
        w = self.words(2 * count).reshape(count, 2).astype(np.uint64)
        hi = w[:, 0] >> np.uint64(5)   # 27 bits
        lo = w[:, 1] >> np.uint64(6)   # 26 bits
        return ((hi << np.uint64(26)) | lo).astype(np.float64) * (1.0 / 9007199254740992.0)

    def gaussian_torus(self, shape, sigma_log2: int) -> np.ndarray:
        """Discretised Gaussian noise on the 32-bit torus: rint(sigma*2^32*z) mod 2^32."""
        shape = tuple(np.atleast_1d(shape)) if not isinstance(shape, tuple) else shape
        cnt = int(np.prod(shape))
        u1 = self.unit_doubles(cnt)
        u2 = self.unit_doubles(cnt)
        z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
        e = np.rint(z * float(2.0 ** (32 + sigma_log2))).astype(np.int64)
        return (e & 0xFFFFFFFF).astype(np.uint32).reshape(shape)

    def uniform_int(self, count: int, lo: int, hi: int) -> np.ndarray:
        """`count` integers uniform in [lo, hi) by 64-bit multiply-shift (bias < 2^-32 * range)."""
        w = self.words(2 * count).reshape(count, 2).astype(np.uint64)
        x = (w[:, 0] << np.uint64(32)) | w[:, 1]
        span = hi - lo
        # floor(x * span / 2^64) computed without overflow via splitting x
        xh = x >> np.uint64(32)
        xl = x & np.uint64(0xFFFFFFFF)
        r = (xh * np.uint64(span) + ((xl * np.uint64(span)) >> np.uint64(32))) >> np.uint64(32)
        return r.astype(np.int64) + lo


# ---------------------------------------------------------------------------
# Random material for key generation and encryption.  Which arithmetic turns
# these numbers into keys and ciphertexts lives elsewhere (the CUDA library's
# client code and, independently, the oracle).
# ---------------------------------------------------------------------------

@dataclass
class KeyMaterial:
    n: int
    N: int
    l: int
    ks_t: int
    ks_base_bits: int
    s: np.ndarray        # [n] LWE key bits
    K: np.ndarray        # [N] TRLWE key bits (k = 1)
    bk_a: np.ndarray     # [n][2l][N] uniform mask polynomials of the TRGSW rows
    bk_e: np.ndarray     # [n][2l][N] Gaussian noise (sigma_BK)
    ksk_a: np.ndarray    # [N][t][base][n] uniform masks of the key-switch rows
    ksk_e: np.ndarray    # [N][t][base] Gaussian noise (sigma_KS)


def key_material(seed: int = MASTER_SEED, *, n=630, N=1024, l=3, ks_t=8, ks_base_bits=2,
                 sigma_bk_log2=SIGMA_BK_LOG2, sigma_ks_log2=SIGMA_KS_LOG2,
                 noiseless: bool = False) -> KeyMaterial:
    """All random numbers key generation consumes, from stream 1 (keys)."""
    base = 1 << ks_base_bits
    st = Stream(seed, STREAM_KEYS, 0)
    s = st.bits(n)
    K = st.bits(N)
    bk_a = Stream(seed, STREAM_KEYS, 1).torus((n, 2 * l, N))
    ksk_a = Stream(seed, STREAM_KEYS, 3).torus((N, ks_t, base, n))
    if noiseless:
        bk_e = np.zeros((n, 2 * l, N), dtype=np.uint32)
        ksk_e = np.zeros((N, ks_t, base), dtype=np.uint32)
    else:
        bk_e = Stream(seed, STREAM_KEYS, 2).gaussian_torus((n, 2 * l, N), sigma_bk_log2)
        ksk_e = Stream(seed, STREAM_KEYS, 4).gaussian_torus((N, ks_t, base), sigma_ks_log2)
    return KeyMaterial(n, N, l, ks_t, ks_base_bits, s, K, bk_a, bk_e, ksk_a, ksk_e)


@dataclass
class LweMaterial:
    a: np.ndarray   # [count][n] uniform masks
    e: np.ndarray   # [count] Gaussian noise (sigma_LWE)


def lwe_material(count: int, n: int = 630, *, seed: int = MASTER_SEED, stream: int = STREAM_QUERY,
                 substream: int = 0, sigma_log2: int = SIGMA_LWE_LOG2,
                 noiseless: bool = False) -> LweMaterial:
    st = Stream(seed, stream, substream)
    a = st.torus((count, n))
    if noiseless:
        e = np.zeros(count, dtype=np.uint32)
    else:
        e = Stream(seed, stream, substream + 0x10000).gaussian_torus((count,), sigma_log2)
    return LweMaterial(a, e)


def value_bits(values, width: int) -> np.ndarray:
    """LSB-first bit decomposition of unsigned integers (bit i = (v >> i) & 1)."""
    v = np.asarray(values, dtype=np.uint64).reshape(-1)
    return ((v[:, None] >> np.arange(width, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint32)


# ---------------------------------------------------------------------------
# Plaintext databases and queries shaped like the paper's workloads.
# ---------------------------------------------------------------------------

def distinct_u32(st: Stream, count: int, width: int = 32) -> np.ndarray:
    """`count` distinct values uniform in [0, 2^width), in draw order."""
    out = []
    seen = set()
    mask = (1 << width) - 1
    while len(out) < count:
        for w in st.words(max(16, 2 * (count - len(out)))):
            v = int(w) & mask
            if v not in seen:
                seen.add(v)
                out.append(v)
                if len(out) == count:
                    break
    return np.array(out, dtype=np.uint32)


def idm_workload(D: int, width: int, *, seed: int = MASTER_SEED, substream: int = 0,
                 payload: bool = False, distinct: bool = False):
    """Identifier matching: a query id, D plaintext ids with the query planted once,
    and (optionally) a 32-bit payload per entry."""
    st = Stream(seed, STREAM_DB, substream)
    mask = (1 << width) - 1
    if distinct:
        ids = distinct_u32(st, D, width)
    else:
        ids = (st.words(D) & np.uint32(mask)).astype(np.uint32)
    planted = int(st.uniform_int(1, 0, D)[0])
    query = int(ids[planted])
    pay = st.words(D) if payload else None
    return dict(query=query, ids=ids, planted=planted, payload=pay, width=width)


def intv_workload(D: int, *, seed: int = MASTER_SEED, substream: int = 0):
    """Interval validation: query point (x, y) uniform u32; D rectangles with
    lo < hi per axis (two uniform draws, sorted; redrawn when equal)."""
    st = Stream(seed, STREAM_DB, substream)
    q = st.words(2)
    rects = np.zeros((D, 4), dtype=np.uint32)
    for d in range(D):
        for ax in range(2):
            while True:
                u, v = (int(w) for w in st.words(2))
                if u != v:
                    break
            rects[d, 2 * ax] = min(u, v)
            rects[d, 2 * ax + 1] = max(u, v)
    return dict(x=int(q[0]), y=int(q[1]), rects=rects)


def cov_workload(D: int, *, seed: int = MASTER_SEED, substream: int = 0):
    """Coordinate validation: a query cell (x, y) on the 2^16 x 2^16 grid, D
    uniform cells packed (y << 16) | x, the query planted once."""
    st = Stream(seed, STREAM_DB, substream)
    cells = st.words(D)
    planted = int(st.uniform_int(1, 0, D)[0])
    return dict(cell=int(cells[planted]), cells=cells, planted=planted)


def log_uniform_sizes(count: int, lo: int, hi: int, *, seed: int = MASTER_SEED, substream: int = 0):
    """floor(lo * (hi/lo)^U) with U uniform in [0, 1)."""
    st = Stream(seed, STREAM_DB, substream)
    u = st.unit_doubles(count)
    return np.floor(lo * np.power(hi / lo, u)).astype(np.int64)


def poisson_arrivals(count: int, rate_per_s: float, *, seed: int = MASTER_SEED, substream: int = 0):
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    st = Stream(seed, STREAM_ARRIVALS, substream)
    u = st.unit_doubles(count)
    return np.cumsum(-np.log1p(-u) / rate_per_s)
