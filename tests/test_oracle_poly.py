"""Pins of the oracle's ring arithmetic in Z_{2^32}[X]/(X^N+1).

The independent reference is Kronecker substitution: both polynomials are
packed into Python integers, multiplied with Python's big-integer product, and
the exact integer coefficients are unpacked and folded by X^N = -1."""
import numpy as np
import pytest

import oracle

M32 = (1 << 32) - 1


def kronecker_negacyclic(a, b):
    N = len(a)
    slot = 80  # every exact product coefficient is < N * 2^64 < 2^80
    A = sum(int(x) << (slot * i) for i, x in enumerate(a))
    B = sum(int(x) << (slot * i) for i, x in enumerate(b))
    C = A * B
    mask = (1 << slot) - 1
    c = [(C >> (slot * k)) & mask for k in range(2 * N)]
    return np.array([(c[k] - c[k + N]) & M32 for k in range(N)], dtype=np.uint32)


def monomial(e, N):
    """X^e as a polynomial in the ring (X^N = -1)."""
    e %= 2 * N
    p = np.zeros(N, dtype=np.uint32)
    if e < N:
        p[e] = 1
    else:
        p[e - N] = M32
    return p


@pytest.mark.parametrize("N", [8, 64, 1024])
def test_schoolbook_equals_kronecker(N):
    rng = np.random.default_rng(N)
    cases = [rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32) for _ in range(2)]
    cases.append(np.full(N, M32, dtype=np.uint32))
    edge = np.zeros(N, dtype=np.uint32); edge[N - 1] = 0x80000000
    cases.append(edge)
    for a in cases:
        for b in cases:
            assert np.array_equal(oracle.poly_mul_schoolbook(a, b), kronecker_negacyclic(a, b))


@pytest.mark.parametrize("N", [16, 64, 256, 1024])
def test_karatsuba_equals_kronecker(N):
    rng = np.random.default_rng(100 + N)
    for _ in range(3):
        a = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(-64, 64, N).astype(np.int64).astype(np.uint32)  # digit-like operand
        assert np.array_equal(oracle.poly_mul_karatsuba(a, b), kronecker_negacyclic(a, b))
        assert np.array_equal(oracle.poly_mul_karatsuba(a, a), kronecker_negacyclic(a, a))
    full = np.full(N, M32, dtype=np.uint32)
    assert np.array_equal(oracle.poly_mul_karatsuba(full, full), kronecker_negacyclic(full, full))


def test_monomial_rotation_exhaustive_toy():
    N = 8
    rng = np.random.default_rng(1)
    p = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    neg = (np.uint32(0) - p).astype(np.uint32)
    assert np.array_equal(oracle.poly_mul_xe(p, N), neg)          # X^N = -1
    assert np.array_equal(oracle.poly_mul_xe(p, 2 * N), p)        # X^2N = 1
    for e1 in range(-2 * N, 2 * N + 1):
        r1 = oracle.poly_mul_xe(p, e1)
        assert np.array_equal(r1, kronecker_negacyclic(p, monomial(e1, N)))
        for e2 in range(-2 * N, 2 * N + 1):
            assert np.array_equal(oracle.poly_mul_xe(r1, e2), oracle.poly_mul_xe(p, e1 + e2))


def test_monomial_rotation_paper_size():
    N = 1024
    rng = np.random.default_rng(2)
    p = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    for e in [0, 1, 511, 1023, 1024, 1025, 2047, -1, -1024, 3000]:
        assert np.array_equal(oracle.poly_mul_xe(p, e), kronecker_negacyclic(p, monomial(e, N)))
