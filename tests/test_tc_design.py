"""Host model of the exact tensor-core external product (VP_PATH_TENSOR_F16),
checked against the oracle's ring product.

The tensor-core path computes out_j[m] = sum over six digit rows r and
k < 1024 of T_{r,j}[m][k] d_r[k] mod 2^32, where T is the negacyclic
Toeplitz matrix of a key polynomial (T[m][k] = BK[m-k], or -BK[m-k+N] mod
2^32 when m < k), on fp16 operands with fp32 accumulation.  It is exact
because (i) every 32-bit key entry is split into four balanced base-256
limbs b_l in [-128, 127] with sum_l b_l 2^(8l) = entry (mod 2^32; the top
limb drops the carry 2^32), (ii) limbs and digits (|d| <= 64) are small
integers that fp16 holds exactly, and (iii) one digit row's 1,024 products
are each at most 2^13 in magnitude, so every partial sum of an fp32
accumulator is an integer of magnitude <= 2^23 < 2^24 and no summation order
rounds.  This model restates the limb split and accumulates in numpy
float32 in K = 16 blocks taken in a random order (the MMA's K), asserting
each accumulator equals the exact int64 sum, and recombines sum_l S_l << 8l
mod 2^32 -- at random inputs and at the extremes (every limb -128 against
digits -64 reaches the 2^23 bound) -- against the oracle's schoolbook product.
It shares no code with the kernels, which the GPU tests compare with the
oracle bit for bit.
"""
import numpy as np
import pytest

import oracle

N = 1024
M32 = (1 << 32) - 1


def limbs(w):
    """Balanced base-256 limbs of uint32 words: four int arrays in [-128, 127]."""
    x = np.asarray(w, dtype=np.int64)
    out = []
    for _ in range(4):
        d = ((x + 128) & 255) - 128
        out.append(d)
        x = (x - d) >> 8
    return out


def toeplitz(bk_row):
    """The negacyclic Toeplitz matrix of one key polynomial, uint32 entries."""
    m = np.arange(N)[:, None]
    k = np.arange(N)[None, :]
    e = m - k
    v = bk_row.astype(np.uint64)[np.where(e >= 0, e, e + N)]
    return np.where(e >= 0, v, (np.uint64(1 << 32) - v) & np.uint64(M32)).astype(np.uint32)


def tc_product(digits, bk, rng):
    """digits int64[6][N], bk uint32[6][2][N] -> out uint32[2][N] the way the tensor-core path computes it."""
    out = np.zeros((2, N), dtype=np.uint64)
    for j in range(2):
        for r in range(6):
            T = toeplitz(bk[r][j])
            d16 = digits[r].astype(np.float16)
            assert np.array_equal(d16.astype(np.int64), digits[r])
            for l, b in enumerate(limbs(T)):
                assert b.min() >= -128 and b.max() <= 127
                b16 = b.astype(np.float16)
                assert np.array_equal(b16.astype(np.int64), b)
                acc = np.zeros(N, dtype=np.float32)
                for kb in rng.permutation(N // 16):
                    blk = slice(16 * kb, 16 * kb + 16)
                    part = (b16[:, blk].astype(np.float32) * d16[blk].astype(np.float32)).astype(np.float32)
                    for c in range(16):              # one fp32 add per term
                        acc = (acc + part[:, c]).astype(np.float32)
                exact = b @ digits[r]
                assert np.abs(exact).max() <= 1 << 23
                assert np.array_equal(acc.astype(np.int64), exact)
                out[j] += (acc.astype(np.int64) << (8 * l)).astype(np.uint64) & np.uint64(M32)
    return (out & np.uint64(M32)).astype(np.uint32)


def exact(digits, bk):
    out = np.zeros((2, N), dtype=np.uint32)
    for j in range(2):
        for r in range(6):
            out[j] = out[j] + oracle.poly_mul_schoolbook(digits[r].astype(np.int64).astype(np.uint32), bk[r][j])
    return out


def test_limb_split_reconstructs_every_word_class():
    words = np.array([0, 1, 127, 128, 255, 256, 0x7F7F7F7F, 0x7F7F7F80, 0x80808080, 0x80000000, M32, 0xDEADBEEF],
                     dtype=np.uint64)
    rng = np.random.default_rng(7)
    words = np.concatenate([words, rng.integers(0, 1 << 32, size=4096, dtype=np.uint64)])
    ls = limbs(words)
    for b in ls:
        assert b.min() >= -128 and b.max() <= 127
    rec = sum(b << (8 * l) for l, b in enumerate(ls))
    assert np.array_equal(rec & M32, words.astype(np.int64))
    assert [int(b[7]) for b in ls] == [-128] * 4          # 0x7F7F7F80: every limb at the bound


def test_model_equals_the_oracle_product_on_random_inputs():
    rng = np.random.default_rng(20250615)
    d = rng.integers(-64, 64, size=(6, N), dtype=np.int64)
    bk = rng.integers(0, 1 << 32, size=(6, 2, N), dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(tc_product(d, bk, rng), exact(d, bk))


@pytest.mark.parametrize("digit, word", [(-64, 0x7F7F7F80), (63, 0x80808080), (-64, M32)])
def test_extreme_limbs_and_digits_stay_exact(digit, word):
    """Constant rows: limbs at -128 against digits -64 make every product
    2^13 and a full row 2^23, the bound of exact fp32 accumulation."""
    rng = np.random.default_rng(3)
    d = np.full((6, N), digit, dtype=np.int64)
    bk = np.full((6, 2, N), word, dtype=np.uint32)
    assert np.array_equal(tc_product(d, bk, rng), exact(d, bk))
