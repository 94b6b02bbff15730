"""Property tests of the launch scheduler through the host dry run
(velopir_plan_query): for random database sizes, contents, wave sizes and
aggregation fan-ins, every scheduled program answers its plaintext predicate
(Alg. InterValid, CoV, IdM with the Section 5 HomSum or the fan-in-g tree),
issues exactly the circuit's bootstraps, launches whole waves (or all that is
ready), and never reads a pool slot after its reuse (the dry run reports
that as ERR_PLAN)."""
import numpy as np
import pytest

from paper_2506_12761_gb300 import velopir as vp

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies
given, settings = hypothesis.given, hypothesis.settings

WAVES = st.sampled_from([0, 1, 7, 48, 1824])


def bits(v, n):
    return np.array([(int(v) >> i) & 1 for i in range(n)], dtype=np.uint32)


def fanin_nodes(D, g):
    nodes, k = 0, 1
    while k < D:
        nodes += sum(1 for i in range(0, D, g * k) if sum(1 for q in range(g) if i + q * k < D) >= 2)
        k *= g
    return nodes


def whole_waves(sizes, wave):
    return not wave or all(s % wave == 0 or s < wave for s in sizes)


@settings(max_examples=150, deadline=None)
@given(D=st.integers(1, 60), wave=WAVES, seed=st.integers(0, 2**31))
def test_intv_random(D, wave, seed):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2**32, size=(D, 2, 2), dtype=np.uint64)
    x, y = (int(v) for v in rng.integers(0, 2**32, size=2, dtype=np.uint64))
    u[rng.random(D) < 0.3, 0, :] = [x, x + 1]          # plant hits and boundary cases on x
    u = np.minimum(np.sort(u, axis=2), 2**32 - 1)
    rects = u.reshape(D, 4).astype(np.uint32)
    r = rects.astype(np.int64)
    want = ((r[:, 0] <= x) & (x < r[:, 1]) & (r[:, 2] <= y) & (y < r[:, 3])).astype(np.uint32)
    out, sizes = vp.velopir_plan_query(vp.VP_QUERY_INTV, rects, D, bits(x, 32), bits(y, 32), wave=wave)
    assert np.array_equal(out, want)
    assert sum(sizes) == 131 * D and whole_waves(sizes, wave)


@settings(max_examples=150, deadline=None)
@given(D=st.integers(1, 200), wave=WAVES, seed=st.integers(0, 2**31), near=st.integers(0, 31))
def test_cov_random(D, wave, seed, near):
    rng = np.random.default_rng(seed)
    cells = rng.integers(0, 2**32, size=D, dtype=np.uint64).astype(np.uint32)
    q = int(cells[rng.integers(D)])
    cells[rng.integers(D)] = q ^ (1 << near)            # one bit away
    out, sizes = vp.velopir_plan_query(vp.VP_QUERY_COV, cells, D, bits(q, 32), wave=wave)
    assert np.array_equal(out, (cells == q).astype(np.uint32))
    assert sum(sizes) == 31 * D and whole_waves(sizes, wave)


@settings(max_examples=150, deadline=None)
@given(D=st.integers(1, 300), wave=WAVES, seed=st.integers(0, 2**31), fanin=st.sampled_from([2, 3, 4, 5, 8]),
       pbits=st.integers(1, 32), hit=st.booleans())
def test_idm_payload_random(D, wave, seed, fanin, pbits, hit):
    rng = np.random.default_rng(seed)
    ids = rng.choice(2**32, size=D, replace=False).astype(np.uint32)
    pay = rng.integers(0, 2**32, size=D, dtype=np.uint64).astype(np.uint32)
    k = int(rng.integers(D))
    q = int(ids[k]) if hit else int(rng.integers(0, 2**32))
    want = 0
    for i in np.flatnonzero(ids == q):
        want ^= int(pay[i])
    out, sizes = vp.velopir_plan_query(vp.VP_QUERY_IDM, ids, D, bits(q, 32), wave=wave, id_bits=32, payload=pay,
                                       payload_bits=pbits, agg_fanin=0 if fanin == 2 else fanin)
    assert np.array_equal(out, bits(want, pbits))
    assert sum(sizes) == 31 * D + pbits * fanin_nodes(D, fanin) and whole_waves(sizes, wave)
