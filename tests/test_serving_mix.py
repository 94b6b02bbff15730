"""The serving benchmark's workload generator, on the CPU: the 40/30/30
IntV/CoV/IdM mix with log-uniform database sizes, the Poisson arrivals, and
the bootstrap counts that turn the measured bootstraps/s into queries/s,
which must equal what the scheduler actually issues (velopir_plan_query's
blind rotations per launch, summed)."""
import numpy as np
import pytest

from paper_2506_12761_gb300 import serve_bench, synth
from paper_2506_12761_gb300 import velopir as vp

SEED = synth.MASTER_SEED


def test_mix_shares_and_size_ranges():
    shapes = [serve_bench.query_shape(100000 + q, SEED) for q in range(2000)]
    kinds = np.array([k for k, _ in shapes])
    shares = [float(np.mean(kinds == k)) for k in range(3)]
    assert abs(shares[0] - 0.4) < 0.035 and abs(shares[1] - 0.3) < 0.035 and abs(shares[2] - 0.3) < 0.035
    for k, (lo, hi) in enumerate([(256, 4096), (256, 16384), (1024, 65536)]):
        D = np.array([d for kk, d in shapes if kk == k])
        assert D.min() >= lo and D.max() < hi
        # log-uniform: half of the sizes lie below the geometric mean of the range
        assert abs(float(np.mean(D < np.sqrt(lo * hi))) - 0.5) < 0.06


def test_poisson_arrivals_have_the_offered_rate():
    t = synth.poisson_arrivals(20000, 0.25, substream=3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(float(np.mean(gaps)) - 4.0) < 0.1            # 1 / rate
    assert abs(float(np.std(gaps)) - 4.0) < 0.2             # exponential: std = mean


def _bits(v, n):
    return np.array([(int(v) >> i) & 1 for i in range(n)], dtype=np.uint32)


@pytest.mark.parametrize("kind, D, fanin", [(0, 37, 2), (1, 300, 2), (2, 129, 2), (2, 129, 8), (2, 1000, 4)])
def test_bootstrap_counts_equal_the_scheduled_rotations(kind, D, fanin):
    rng = np.random.default_rng(D + fanin)
    if kind == 0:
        u = np.sort(rng.integers(0, 2**32, size=(D, 2, 2), dtype=np.uint64), axis=2)
        db = u.reshape(D, 4).astype(np.uint32)
        _, sizes = vp.velopir_plan_query(vp.VP_QUERY_INTV, db, D, _bits(5, 32), _bits(7, 32), wave=1824)
    elif kind == 1:
        db = rng.integers(0, 2**32, size=D, dtype=np.uint64).astype(np.uint32)
        _, sizes = vp.velopir_plan_query(vp.VP_QUERY_COV, db, D, _bits(int(db[0]), 32), wave=1824)
    else:
        db = rng.choice(2**32, size=D, replace=False).astype(np.uint32)
        pay = rng.integers(0, 2**32, size=D, dtype=np.uint64).astype(np.uint32)
        _, sizes = vp.velopir_plan_query(vp.VP_QUERY_IDM, db, D, _bits(int(db[3]), 32), wave=1824, id_bits=32,
                                         payload=pay, payload_bits=32, agg_fanin=0 if fanin == 2 else fanin)
    assert sum(sizes) == serve_bench.bootstraps_of(kind, D, fanin)
