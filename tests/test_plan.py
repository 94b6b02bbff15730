"""The launch scheduler, checked on the CPU through velopir_plan_query.

The dry run executes the scheduled gate program on noiseless plaintext
phases with the device's pool-slot reuse, so a dependency the scheduler
breaks (a gate placed in the launch of, or before, a gate it reads) or a
pool slot reused too early either makes the answer wrong or is reported as
ERR_PLAN.  Answers are compared with the plaintext predicates of the modes
(Alg. InterValid, CoV, IdM with HomSum aggregation of Section 5)."""
import numpy as np
import pytest

from paper_2506_12761_gb300 import velopir as vp

WAVES = (0, 48, 64, 1824)


def bits(v, n):
    return np.array([(int(v) >> i) & 1 for i in range(n)], dtype=np.uint32)


def intv_case(D, seed):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2**32, size=(D, 4), dtype=np.uint64)
    lo = np.minimum(u[:, [0, 2]], u[:, [1, 3]])
    hi = np.maximum(u[:, [0, 2]], u[:, [1, 3]])
    x, y = (int(v) for v in rng.integers(0, 2**32, size=2, dtype=np.uint64))
    # plant hits and near misses on the bounds
    lo[: D // 4, 0], hi[: D // 4, 0] = x, x + 1
    lo[D // 4: D // 2, 1] = y + 1
    rects = np.stack([lo[:, 0], hi[:, 0], lo[:, 1], hi[:, 1]], axis=1).astype(np.uint64)
    rects = np.minimum(rects, 2**32 - 1).astype(np.uint32)
    r = rects.astype(np.int64)
    want = ((r[:, 0] <= x) & (x < r[:, 1]) & (r[:, 2] <= y) & (y < r[:, 3])).astype(np.uint32)
    return rects, bits(x, 32), bits(y, 32), want


def launches_are_waves(sizes, wave, total):
    assert sum(sizes) == total
    if wave:
        # a launch is a whole number of waves, or all that was ready when
        # less than a wave was
        assert all(s % wave == 0 or s < wave for s in sizes), sizes


@pytest.mark.parametrize("wave", WAVES)
def test_intv_plan_answers_the_predicate(wave):
    D = 200
    rects, bx, by, want = intv_case(D, 3)
    out, sizes = vp.velopir_plan_query(vp.VP_QUERY_INTV, rects, D, bx, by, wave=wave)
    assert np.array_equal(out, want)
    assert 0 < want.sum() < D
    launches_are_waves(sizes, wave, 131 * D)


def test_wave_filling_shortens_the_schedule_in_waves():
    """IntV D = 1,024 at 12 bootstraps per SM: 34 ASAP layers need 2.25 waves
    each (3 launched waves per 4,096-gate layer); the wave-filled schedule
    needs 74 waves in total, all full but the last."""
    D = 1024
    rects, bx, by, want = intv_case(D, 4)
    wave = 152 * 12
    out0, asap = vp.velopir_plan_query(vp.VP_QUERY_INTV, rects, D, bx, by, wave=0)
    out1, filled = vp.velopir_plan_query(vp.VP_QUERY_INTV, rects, D, bx, by, wave=wave)
    assert np.array_equal(out0, want) and np.array_equal(out1, want)
    assert len(asap) == 34 and asap[0] == 4096
    waves = lambda sizes: sum(-(-s // wave) for s in sizes)
    assert waves(asap) == 32 * 3 + 2 + 1
    assert waves(filled) == -(-131 * D // wave) == 74


@pytest.mark.parametrize("wave", WAVES)
def test_cov_plan_answers_equality(wave):
    rng = np.random.default_rng(5)
    D = 150
    cells = rng.integers(0, 2**32, size=D, dtype=np.uint64).astype(np.uint32)
    q = int(cells[17])
    cells[60] = q ^ 1          # one bit off in x
    cells[61] = q ^ (1 << 31)  # one bit off in y
    out, sizes = vp.velopir_plan_query(vp.VP_QUERY_COV, cells, D, bits(q, 32), wave=wave)
    assert np.array_equal(out, (cells == q).astype(np.uint32))
    launches_are_waves(sizes, wave, 31 * D)


@pytest.mark.parametrize("wave", WAVES)
def test_idm_payload_aggregation_plan(wave):
    rng = np.random.default_rng(6)
    D = 77
    ids = rng.choice(2**32, size=D, replace=False).astype(np.uint32)
    pay = rng.integers(0, 2**32, size=D, dtype=np.uint64).astype(np.uint32)
    q = int(ids[40])
    out, sizes = vp.velopir_plan_query(vp.VP_QUERY_IDM, ids, D, bits(q, 32), wave=wave, id_bits=32,
                                       payload=pay, payload_bits=32)
    assert np.array_equal(out, bits(pay[40], 32))
    launches_are_waves(sizes, wave, 31 * D + 32 * (D - 1))
    miss, _ = vp.velopir_plan_query(vp.VP_QUERY_IDM, ids, D, bits(q ^ 4, 32), wave=wave, id_bits=32,
                                    payload=pay, payload_bits=32)
    assert not miss.any() or (q ^ 4) in set(ids.tolist())


@pytest.mark.parametrize("id_bits", [1, 5, 8, 32])
def test_idm_match_bits_plan(id_bits):
    rng = np.random.default_rng(id_bits)
    D = 40
    ids = rng.integers(0, 2**id_bits, size=D, dtype=np.uint64).astype(np.uint32)
    q = int(ids[3])
    out, _ = vp.velopir_plan_query(vp.VP_QUERY_IDM, ids, D, bits(q, id_bits), wave=16, id_bits=id_bits)
    assert np.array_equal(out, (ids == q).astype(np.uint32))


def test_plan_rejects_bad_arguments():
    cells = np.zeros(4, dtype=np.uint32)
    with pytest.raises(vp.VelopirError):
        vp.velopir_plan_query(vp.VP_QUERY_COV, cells, 0, bits(0, 32))
    with pytest.raises(vp.VelopirError):
        vp.velopir_plan_query(vp.VP_QUERY_IDM, cells, 4, bits(0, 32), id_bits=33)
    with pytest.raises(vp.VelopirError):
        vp.velopir_plan_query(vp.VP_QUERY_INTV, np.zeros((4, 4), np.uint32), 4, bits(0, 32), None)
    with pytest.raises(vp.VelopirError):
        vp.velopir_plan_query(7, cells, 4, bits(0, 32))


# ---- the encrypted-database circuits (the *_encdb calls) ----

def xor_of(values, valid):
    acc = 0
    for v, ok in zip(values, valid):
        acc ^= int(v) if ok else 0
    return acc


@pytest.mark.parametrize("wave", [0, 64])
def test_intv_encdb_plan_at_the_papers_width(wave):
    """l_I = 16 with encrypted bounds and a 9-bit encrypted payload (covid-kor's
    shape, M larger): the HomCompLeOPT MUX ripple, HomBitwiseAND and HomSum."""
    rng = np.random.default_rng(21)
    D, l = 40, 16
    u = rng.integers(0, 1 << l, size=(D, 4))
    x, y = 40000, 1234
    lo, hi = np.minimum(u[:, [0, 2]], u[:, [1, 3]]), np.maximum(u[:, [0, 2]], u[:, [1, 3]])
    lo[::5], hi[::5] = [x - 3, y], [x + 1, y + 1]
    rects = np.stack([lo[:, 0], hi[:, 0], lo[:, 1], hi[:, 1]], axis=1).astype(np.uint32)
    valid = (rects[:, 0] <= x) & (x < rects[:, 1]) & (rects[:, 2] <= y) & (y < rects[:, 3])
    out, sizes = vp.velopir_plan_query(vp.VP_PLAN_INTV_ENCDB, rects, D, bits(x, l), bits(y, l), wave=wave, id_bits=l)
    assert np.array_equal(out, valid.astype(np.uint32)) and 0 < valid.sum() < D
    launches_are_waves(sizes, wave, (12 * l + 3) * D)
    pay = rng.integers(0, 1 << 9, size=D).astype(np.uint32)
    agg, sizes = vp.velopir_plan_query(vp.VP_PLAN_INTV_ENCDB, rects, D, bits(x, l), bits(y, l), wave=wave, id_bits=l,
                                       payload=pay, payload_bits=9)
    assert np.array_equal(agg, bits(xor_of(pay, valid), 9))
    launches_are_waves(sizes, wave, (12 * l + 3) * D + 9 * D + 9 * (D - 1))


def test_encdb_comparator_boundaries_exhaustive():
    """Every (bound, point) pair at l = 4 through the encrypted comparators:
    rectangles [a, b) x [0, 15) with the point on and around the bounds."""
    l = 4
    for x in range(16):
        rects = np.array([[a, b, 0, 15] for a in range(16) for b in range(16)], dtype=np.uint32)
        out, _ = vp.velopir_plan_query(vp.VP_PLAN_INTV_ENCDB, rects, len(rects), bits(x, l), bits(3, l),
                                       wave=0, id_bits=l)
        want = ((rects[:, 0] <= x) & (x < rects[:, 1])).astype(np.uint32)
        assert np.array_equal(out, want), x


@pytest.mark.parametrize("wave", [0, 48])
def test_cov_and_idm_encdb_plans(wave):
    rng = np.random.default_rng(22)
    w = 16
    cells = rng.integers(0, 1 << 32, size=30, dtype=np.uint64).astype(np.uint32)
    q = int(cells[11])
    cells[12] = q ^ (1 << 20)
    out, _ = vp.velopir_plan_query(vp.VP_PLAN_COV_ENCDB, cells, 30, bits(q, 2 * w), wave=wave, id_bits=w)
    assert np.array_equal(out, (cells == q).astype(np.uint32))
    ids = rng.choice(1 << 16, size=50, replace=False).astype(np.uint32)
    pay = rng.integers(0, 1 << 32, size=50, dtype=np.uint64).astype(np.uint32)
    agg, sizes = vp.velopir_plan_query(vp.VP_PLAN_IDM_ENCDB, ids, 50, bits(int(ids[7]), 16), wave=wave, id_bits=16,
                                       payload=pay, payload_bits=32)
    assert np.array_equal(agg, bits(int(pay[7]), 32))
    launches_are_waves(sizes, wave, 31 * 50 + 32 * 50 + 32 * 49)
    with pytest.raises(vp.VelopirError):
        vp.velopir_plan_query(vp.VP_PLAN_COV_ENCDB, cells, 30, bits(q, 34), id_bits=17)


def test_batch_of_uneven_queries_in_chunked_launch_order():
    """velopir_query_batch's merged program over many queries of all three
    modes (uneven sizes), with wave-filling, executed in the device's order
    with launches split into small chunks: every query's answer is its
    plaintext predicate and no slot is read after reuse."""
    rng = np.random.default_rng(31)
    qs, want = [], []
    for k in range(12):
        mode = k % 3
        D = int(rng.integers(20, 400))
        if mode == 0:
            rects, bx, by, w = intv_case(D, 100 + k)
            qs.append(dict(kind=vp.VP_QUERY_INTV, db=rects, D=D, bits_a=bx, bits_b=by))
            want.append(w)
        elif mode == 1:
            cells = rng.integers(0, 1 << 32, size=D, dtype=np.uint64).astype(np.uint32)
            q = int(cells[D // 2])
            qs.append(dict(kind=vp.VP_QUERY_COV, db=cells, D=D, bits_a=bits(q, 32)))
            want.append((cells == q).astype(np.uint32))
        else:
            ids = rng.choice(1 << 20, size=D, replace=False).astype(np.uint32)
            pay = rng.integers(0, 1 << 32, size=D, dtype=np.uint64).astype(np.uint32)
            qs.append(dict(kind=vp.VP_QUERY_IDM, db=ids, D=D, bits_a=bits(int(ids[3]), 20), id_bits=20,
                           payload=pay, payload_bits=32))
            want.append(np.array(bits(int(pay[3]), 32), dtype=np.uint32))
    for wave, chunk in ((0, 0), (96, 500), (1824, 64)):
        outs, sizes = vp.velopir_plan_batch(qs, wave=wave, chunk_rows=chunk)
        for o, w in zip(outs, want):
            assert np.array_equal(o, w)
        launches_are_waves(sizes, wave, sum(131 * q["D"] if q["kind"] == vp.VP_QUERY_INTV else
                                            31 * q["D"] if q["kind"] == vp.VP_QUERY_COV else
                                            19 * q["D"] + 32 * (q["D"] - 1) for q in qs))


def fanin_nodes(D, g):
    """Bootstraps per payload bit of the fan-in-g XOR tree (groups with >= 2 members)."""
    nodes, k = 0, 1
    while k < D:
        for i in range(0, D, g * k):
            if sum(1 for q in range(g) if i + q * k < D) >= 2:
                nodes += 1
        k *= g
    return nodes


@pytest.mark.parametrize("fanin", [2, 3, 4, 8])
@pytest.mark.parametrize("wave", [0, 64, 1824])
def test_idm_payload_fanin_tree_plan(fanin, wave):
    """The fan-in-g XOR aggregation (one bootstrap of 2 sum c + T((g-1)/4) per
    group) answers the planted entry's payload at ragged sizes, and costs
    31 D + 32 nodes(D, g) bootstraps: (D - 1) / (g - 1) per bit when D is a
    power of g."""
    rng = np.random.default_rng(60 + fanin)
    for D in (1, 2, fanin, fanin + 1, 77, fanin ** 3):
        ids = rng.choice(2**32, size=D, replace=False).astype(np.uint32)
        pay = rng.integers(0, 2**32, size=D, dtype=np.uint64).astype(np.uint32)
        hit = D // 2
        out, sizes = vp.velopir_plan_query(vp.VP_QUERY_IDM, ids, D, bits(int(ids[hit]), 32), wave=wave, id_bits=32,
                                           payload=pay, payload_bits=32, agg_fanin=fanin)
        assert np.array_equal(out, bits(pay[hit], 32)), (D, fanin)
        launches_are_waves(sizes, wave, 31 * D + 32 * fanin_nodes(D, fanin))
    assert fanin_nodes(fanin ** 3, fanin) == (fanin ** 3 - 1) // (fanin - 1)


def test_fanin_tree_in_chunked_batch_order():
    """Several fan-in IdM queries (and a pairwise one) in one merged program,
    wave-filled and split into small chunks: the sums of a layer run before
    its rotations, and no slot is read after reuse."""
    rng = np.random.default_rng(77)
    qs, want = [], []
    for k, (fanin, D) in enumerate(((8, 300), (4, 129), (3, 50), (0, 90))):
        ids = rng.choice(1 << 20, size=D, replace=False).astype(np.uint32)
        pay = rng.integers(0, 1 << 32, size=D, dtype=np.uint64).astype(np.uint32)
        hit = int(rng.integers(0, D))
        qs.append(dict(kind=vp.VP_QUERY_IDM, db=ids, D=D, bits_a=bits(int(ids[hit]), 20), id_bits=20,
                       payload=pay, payload_bits=32, agg_fanin=fanin))
        want.append(bits(int(pay[hit]), 32))
    for wave, chunk in ((0, 0), (96, 37), (1824, 200)):
        outs, _ = vp.velopir_plan_batch(qs, wave=wave, chunk_rows=chunk)
        for o, w in zip(outs, want):
            assert np.array_equal(o, w)


def test_fanin_out_of_range_is_rejected():
    ids = np.arange(8, dtype=np.uint32)
    for bad in (1, 9, -1):
        with pytest.raises(vp.VelopirError):
            vp.velopir_plan_query(vp.VP_QUERY_IDM, ids, 8, bits(3, 32), id_bits=32, payload=ids, payload_bits=32,
                                  agg_fanin=bad)


@pytest.mark.parametrize("fanin", [3, 8])
@pytest.mark.parametrize("wave", [0, 64])
def test_encdb_fanin_tree_plans(fanin, wave):
    """The encrypted-database calls' aggregation with the fan-in-g tree
    (velopir_set_encdb_fanin): each of the three modes answers the XOR of
    the valid entries' payloads and costs its validation bootstraps, one
    AND per payload bit and entry (Alg. HomBitwiseAND), and
    nodes(D, g) per payload bit."""
    rng = np.random.default_rng(90 + fanin)
    l, w, idb, pb = 8, 5, 12, 16
    for D in (1, fanin + 1, 41):
        pay = rng.integers(0, 1 << pb, size=D, dtype=np.uint64).astype(np.uint32)
        agg_cost = pb * D + pb * fanin_nodes(D, fanin)
        # IntV at l bits: entries 0 and D-1 contain the point
        x, y = int(rng.integers(1, 255)), int(rng.integers(1, 255))
        rects = rng.integers(0, 256, size=(D, 4), dtype=np.uint64).astype(np.uint32)
        rects[0] = (x, x + 1, y, y + 1)
        rects[D - 1] = (0, 255, 0, 255)
        r = rects.astype(np.int64)
        valid = (r[:, 0] <= x) & (x < r[:, 1]) & (r[:, 2] <= y) & (y < r[:, 3])
        out, sizes = vp.velopir_plan_query(vp.VP_PLAN_INTV_ENCDB, rects, D, bits(x, l), bits(y, l), wave=wave,
                                           id_bits=l, payload=pay, payload_bits=pb, agg_fanin=fanin)
        assert np.array_equal(out, bits(np.bitwise_xor.reduce(pay[valid]), pb)), (D, fanin)
        launches_are_waves(sizes, wave, (12 * l + 3) * D + agg_cost)
        # CoV: a quarter of the cells equal the query's
        cells = rng.integers(0, 1 << (2 * w), size=D, dtype=np.uint64).astype(np.uint32)
        q = int(cells[0])
        cells[::4] = q
        out, sizes = vp.velopir_plan_query(vp.VP_PLAN_COV_ENCDB, cells, D, bits(q, 2 * w), wave=wave, id_bits=w,
                                           payload=pay, payload_bits=pb, agg_fanin=fanin)
        assert np.array_equal(out, bits(np.bitwise_xor.reduce(pay[cells == q]), pb)), (D, fanin)
        launches_are_waves(sizes, wave, (4 * w - 1) * D + agg_cost)
        # IdM: distinct identifiers, one match
        ids = rng.choice(1 << idb, size=D, replace=False).astype(np.uint32)
        hit = D // 2
        out, sizes = vp.velopir_plan_query(vp.VP_PLAN_IDM_ENCDB, ids, D, bits(int(ids[hit]), idb), wave=wave,
                                           id_bits=idb, payload=pay, payload_bits=pb, agg_fanin=fanin)
        assert np.array_equal(out, bits(int(pay[hit]), pb)), (D, fanin)
        launches_are_waves(sizes, wave, (2 * idb - 1) * D + agg_cost)


def test_fanin_only_where_there_is_an_xor_tree():
    """agg_fanin is accepted for IdM and the encrypted-database kinds, not
    for the plaintext IntV and CoV calls (their outputs are per-entry bits)."""
    rects, bx, by, _ = intv_case(4, 5)
    with pytest.raises(vp.VelopirError):
        vp.velopir_plan_query(vp.VP_QUERY_INTV, rects, 4, bx, by, agg_fanin=4)
    ids = np.arange(4, dtype=np.uint32)
    with pytest.raises(vp.VelopirError):
        vp.velopir_plan_query(vp.VP_PLAN_IDM_ENCDB, ids, 4, bits(1, 8), id_bits=8, payload=ids, payload_bits=8,
                              agg_fanin=9)
