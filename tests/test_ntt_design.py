"""Host model of the exact two-prime NTT external product that the default
blind-rotation kernel computes, checked against the oracle's ring product.

The kernel (one warp per bootstrap) computes, per step, out_j = sum over six
digit polynomials d_r of d_r(X) BK[r][j](X) mod (X^1024 + 1) exactly: a
negacyclic NTT modulo p0 = 167772161 and p1 = 195198977 (Cooley-Tukey
forward, Gentleman-Sande inverse, twiddles psi^(+-brv(k))), Shoup products
with lazy reductions, the first two forward stages of each digit transform
by table lookups, and a Chinese-remainder lift whose sign is decided by one
comparison.  Its correctness rests on value bounds (no reduction in the
forward transform because 22 p < 2^32, six-term pointwise sums below 12 p,
an inverse that reduces every third stage, and |coefficient| < 6 x 1024 x 64
x 2^32 = 2^50.6 < p0 p1 / 2).  This model restates that arithmetic in numpy
(uint64, so an overflow of 32 bits is seen instead of wrapping) and checks
every bound at every stage, on random inputs and on the extreme ones (all
digits -64 or 63, key words 2^32 - 1), then compares the result mod 2^32
with the oracle's schoolbook product.  It shares no code with the kernel;
the kernel itself is compared with the oracle bit for bit in the GPU tests.
"""
import numpy as np
import pytest

import oracle

N = 1024
P = (167772161, 195198977)
M32 = (1 << 32) - 1


def brv10(k):
    return int(f"{k:010b}"[::-1], 2)


def tables(p):
    psi = pow(3, (p - 1) // (2 * N), p)
    assert pow(psi, N, p) == p - 1
    ipsi = pow(psi, p - 2, p)
    fw = np.array([pow(psi, brv10(k), p) for k in range(N)], dtype=np.uint64)
    iw = np.array([pow(ipsi, brv10(k), p) for k in range(N)], dtype=np.uint64)
    return fw, iw


TW = {p: tables(p) for p in P}


SHOUP_COUNT = [0]   # Shoup products executed, for the work count of the roofline


def shoup(x, w, p):
    """x * w mod p in [0, 2p) with ws = floor(w 2^32 / p); x < 2^32 required."""
    x = np.asarray(x, dtype=np.uint64)
    w = np.asarray(w, dtype=np.uint64)
    SHOUP_COUNT[0] += int(np.broadcast(x, w).size)
    assert int(x.max()) <= M32
    ws = (w << np.uint64(32)) // np.uint64(p)
    q = (x * ws) >> np.uint64(32)
    r = (x * w - q * np.uint64(p)) & np.uint64(M32)
    assert int(r.max()) < 2 * p
    assert np.array_equal(r % np.uint64(p), (x * w) % np.uint64(p))
    return r


def red_shoup(x, p):
    """x mod p in [0, 2p) for x < 2^32 (w = 1, pinv = floor(2^32 / p))."""
    x = np.asarray(x, dtype=np.uint64)
    assert int(x.max()) <= M32
    pinv = np.uint64((1 << 32) // p)
    r = x - ((x * pinv) >> np.uint64(32)) * np.uint64(p)
    assert int(r.max()) < 2 * p
    return r


def forward(x, p, s0=0, bound=None):
    """Negacyclic forward transform from stage s0, no reduction: inputs below
    `bound` grow by less than 2p per stage."""
    fw = TW[p][0]
    x = x.copy()
    B = bound if bound is not None else p
    assert int(x.max()) < B
    for s in range(s0, 10):
        m, dist = 1 << s, N >> (s + 1)
        v = x.reshape(m, 2, dist)
        lo, hi = v[:, 0, :].copy(), v[:, 1, :]
        t = shoup(hi, fw[m:2 * m, None], p)
        v[:, 0, :] = lo + t
        v[:, 1, :] = lo - t + np.uint64(2 * p)
        B += 2 * p
        assert int(x.max()) < B and B - 2 * p <= M32
    return x


def digit_stages_by_lookup(d, p):
    """Stages 0 and 1 of a digit polynomial as the kernel's lookups: byte
    b = d + 64, T0[b] = psi^512 d, Ua[b] = psi^256 d, Ub[b] = psi^768 d (mod p)."""
    fw = TW[p][0]
    w512, w256, w768 = int(fw[1]), int(fw[2]), int(fw[3])
    dm = [(int(v) % p) for v in d]
    T0 = lambda i: (w512 * dm[i]) % p
    Ua = lambda i: (w256 * dm[i]) % p
    Ub = lambda i: (w768 * dm[i]) % p
    x = np.zeros(N, dtype=np.uint64)
    for u in range(256):                   # quarter q of the polynomial: u, u+256, u+512, u+768
        xv = int(d[u]) + p                 # b0 + (p - 64) with b0 = d + 64
        t0 = T0(u + 512)
        s0, s1 = xv + t0, xv - t0 + 2 * p
        m0 = Ua(u + 256) + Ub(u + 768)
        m1 = Ub(u + 256) + Ua(u + 768)
        x[u], x[u + 256] = s0 + m0, s0 - m0 + 2 * p
        x[u + 512], x[u + 768] = s1 + m1, s1 - m1 + 2 * p
    assert int(x.max()) < 6 * p
    return x


def inverse2(a, p):
    """Gentleman-Sande inverse: stage k inputs below B = 2p << (k mod 3);
    X = x + y reduced on every third stage, Y = w (x - y + B) mod p below 2p."""
    iw = TW[p][1]
    a = a.copy()
    for k in range(10):
        B = (2 * p) << (k % 3)
        assert int(a.max()) < B
        dist, m = 1 << k, 512 >> k
        v = a.reshape(m, 2, dist)
        lo, hi = v[:, 0, :].copy(), v[:, 1, :].copy()
        X = lo + hi
        if k % 3 == 2:
            X = red_shoup(X, p)
        v[:, 0, :] = X
        v[:, 1, :] = shoup(lo - hi + np.uint64(B), iw[m:2 * m, None], p)
        assert int(a.max()) <= M32
    assert int(a.max()) < 4 * p
    return a


def key_hat(bk_row, p):
    """Transformed key with N^-1 folded in, as the key-transform kernel stores it."""
    k = forward(bk_row.astype(np.uint64) % np.uint64(p), p)
    ninv = pow(N, p - 2, p)
    return (k % np.uint64(p)) * np.uint64(ninv) % np.uint64(p)


def external_product(digits, bk, khat=None):
    """digits int64[6][N] in [-64, 63], bk uint32[6][2][N]: out uint32[2][N] as the kernel computes it."""
    if khat is None:
        khat = {(p, r, j): key_hat(bk[r][j], p) for p in P for r in range(6) for j in range(2)}
    res = {}
    for p in P:
        acc = [np.zeros(N, dtype=np.uint64) for _ in range(2)]
        for r in range(6):
            x = forward(digit_stages_by_lookup(digits[r], p), p, s0=2, bound=6 * p)
            assert int(x.max()) < 22 * p
            for j in range(2):
                acc[j] = acc[j] + shoup(x, khat[(p, r, j)], p)
                assert int(acc[j].max()) < 12 * p
        res[p] = [inverse2(red_shoup(acc[j], p), p) for j in range(2)]
    p0, p1 = P
    crt_inv = pow(p0, p1 - 2, p1)
    Pm32 = np.uint64((p0 * p1) & M32)
    out = np.zeros((2, N), dtype=np.uint32)
    for j in range(2):
        x0 = red_shoup(res[p0][j], p0)
        x0 = np.where(x0 >= p0, x0 - np.uint64(p0), x0)     # [0, 2p) -> [0, p)
        assert int(x0.max()) < p0
        x1 = res[p1][j]
        t = shoup(x1 - x0 + np.uint64(p1), crt_inv, p1)
        t = np.where(t >= p1, t - np.uint64(p1), t)
        lo = (x0 + np.uint64(p0) * t - np.where(t > p1 // 2, Pm32, np.uint64(0))) & np.uint64(M32)
        out[j] = lo.astype(np.uint32)
    return out


def exact(digits, bk):
    """The same product from the oracle's schoolbook ring product mod 2^32."""
    out = np.zeros((2, N), dtype=np.uint32)
    for j in range(2):
        acc = np.zeros(N, dtype=np.uint32)
        for r in range(6):
            acc = acc + oracle.poly_mul_schoolbook(digits[r].astype(np.int64).astype(np.uint32), bk[r][j])
        out[j] = acc
    return out


def test_model_equals_the_oracle_product_on_random_inputs():
    rng = np.random.default_rng(20250615)
    d = rng.integers(-64, 64, size=(6, N), dtype=np.int64)
    bk = rng.integers(0, 1 << 32, size=(6, 2, N), dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(external_product(d, bk), exact(d, bk))


@pytest.mark.parametrize("digit, key", [(-64, M32), (63, M32), (-64, 0x80000000), (63, 1)])
def test_extreme_inputs_keep_every_bound_and_the_crt_sign(digit, key):
    """Constant digits and key words: coefficient N-1 reaches
    |6 x 1024 x 64 x (2^32 - 1)| = 2^50.58, the largest magnitude the CRT
    lift must recover with its one-comparison sign."""
    d = np.full((6, N), digit, dtype=np.int64)
    bk = np.full((6, 2, N), key, dtype=np.uint32)
    got = external_product(d, bk)
    assert np.array_equal(got, exact(d, bk))
    # the exact integer at k = N - 1 is 6 * digit * key * N (every term enters with +1)
    assert int(got[0][N - 1]) == (6 * digit * key * N) & M32


def test_mixed_signs_and_ragged_digits():
    """Alternating extremes in the digits and a key with both extreme and small words."""
    d = np.where(np.arange(N) % 2 == 0, -64, 63)[None, :].repeat(6, axis=0).astype(np.int64)
    d[3, ::7] = 0
    bk = np.full((6, 2, N), M32, dtype=np.uint32)
    bk[:, 1, ::3] = 0
    bk[2, 0, ::5] = 1
    assert np.array_equal(external_product(d, bk), exact(d, bk))


def test_executed_work_matches_the_roofline_count():
    """The Shoup products one external product executes (8 multiplying
    stages of 12 forward digit transforms, the pointwise products, 4 inverse
    transforms and the CRT lift) equal the per-step count behind the
    benchmark's roofline (ntt_model), and the lookups replace exactly the
    first two stages."""
    from paper_2506_12761_gb300 import ntt_model
    rng = np.random.default_rng(11)
    d = rng.integers(-64, 64, size=(6, N), dtype=np.int64)
    bk = rng.integers(0, 1 << 32, size=(6, 2, N), dtype=np.uint64).astype(np.uint32)
    khat = {(p, r, j): key_hat(bk[r][j], p) for p in P for r in range(6) for j in range(2)}
    SHOUP_COUNT[0] = 0
    external_product(d, bk, khat)
    assert SHOUP_COUNT[0] == ntt_model.SHOUP_PER_STEP == 12 * 8 * 512 + 2 * 6 * 2 * N + 4 * 10 * 512 + 2 * N
    assert ntt_model.IMAD_SLOTS_PER_BOOTSTRAP == (4 * ntt_model.SHOUP_PER_STEP + ntt_model.CRT_PER_STEP) * 630
