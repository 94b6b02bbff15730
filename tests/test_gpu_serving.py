"""Multi-query batches (one merged program, optional CUDA-graph replay) and the
continuous-batching serving loop: every result is bit-identical to the
oracle's circuit on the query's own ciphertexts, and to the same query run
alone."""
import numpy as np
import pytest

from gpu_common import as_record, check_trace, encrypt_value_bits, gpu_ctx, make_queries, oracle_out
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def run_alone(ctx, q):
    out = np.zeros_like(q["out"])
    if q["kind"] == vp.VP_QUERY_INTV:
        vp.velopir_interval_query(ctx.h, q["a"], q["b"], q["db"], q["D"], out)
    elif q["kind"] == vp.VP_QUERY_COV:
        vp.velopir_coordinate_query(ctx.h, q["a"], q["db"], q["D"], out)
    elif q.get("fanin", 0):
        vp.velopir_query_batch(ctx.h, [vp.make_query(q["kind"], q["a"], q["db"], q["D"], out, id_bits=q["id_bits"],
                                                     payload=q["payload"], payload_bits=q["payload_bits"],
                                                     agg_fanin=q["fanin"])])
    else:
        vp.velopir_id_match(ctx.h, q["a"], q["id_bits"], q["db"], q["D"], q["payload"], q["payload_bits"], out)
    return out


def test_query_batch_matches_alone_and_oracle(paper_keys):
    ctx, s = gpu_ctx()
    qs = make_queries(s, 3)
    vp.velopir_query_batch(ctx.h, [as_record(q) for q in qs])
    for q in qs:
        assert np.array_equal(q["out"], run_alone(ctx, q))
    for q in qs:
        assert np.array_equal(q["out"], oracle_out(paper_keys, q))


def test_query_batch_graph_replay(paper_keys):
    ctx, s = gpu_ctx()
    qs = make_queries(s, 4, fanin=4)
    r0 = vp.velopir_graph_replays(ctx.h)
    vp.velopir_query_batch(ctx.h, [as_record(q) for q in qs], use_graph=True)
    first = [q["out"].copy() for q in qs]
    for q in qs:
        q["out"][:] = 0
    vp.velopir_query_batch(ctx.h, [as_record(q) for q in qs], use_graph=True)
    assert vp.velopir_graph_replays(ctx.h) == r0 + 1
    for q, f in zip(qs, first):
        assert np.array_equal(q["out"], f)
        assert np.array_equal(q["out"], oracle_out(paper_keys, q))


def test_serving_results_identical_alone_and_in_the_mix(paper_keys):
    """Queries arriving while others are on the GPU are admitted into the
    running layer batches; each result equals the oracle's circuit on the
    query's inputs and the query run alone, and every traced gate of the
    serving steps equals the oracle's."""
    ctx, s = gpu_ctx()
    qs = make_queries(s, 3) + make_queries(s, 4, fanin=4)
    alone = [run_alone(ctx, q) for q in qs]
    vp.velopir_trace_start(ctx.h, 33, 4, 0, 4096)
    tickets = {}
    pending = list(range(len(qs)))
    done = set()
    polls = 0
    # staggered arrivals: one new query every other poll
    while len(done) < len(qs):
        if pending and polls % 2 == 0:
            i = pending.pop(0)
            tickets[i] = vp.velopir_submit(ctx.h, as_record(qs[i]))
        for i, t in list(tickets.items()):
            if i not in done and vp.velopir_poll(ctx.h, t):
                done.add(i)
        polls += 1
        assert polls < 500
    recs = vp.velopir_trace_stop(ctx.h, 4096)
    for q, a in zip(qs, alone):
        assert np.array_equal(q["out"], oracle_out(paper_keys, q))
        assert np.array_equal(q["out"], a)
    assert vp.velopir_queue_depth(ctx.h) == (0, 0)
    check_trace(paper_keys, recs, 64)


def test_serving_admission_respects_memory_budget(paper_keys):
    """A context with a small HBM budget admits queries one at a time but still finishes them all."""
    _, s = gpu_ctx()
    from gpu_common import _state
    km = synth.key_material()
    bk, ksk = vp.velopir_client_keygen(km)
    ctx = vp.Context(0, hbm_budget_bytes=700 << 20)
    vp.velopir_load_cloud_key(ctx.h, bk, ksk)
    qs = make_queries(s, 3)
    alone = [run_alone(_state["ctx"], q) for q in qs]
    ts = [vp.velopir_submit(ctx.h, as_record(q)) for q in qs]
    left = set(range(len(qs)))
    for _ in range(400):
        for i in list(left):
            if vp.velopir_poll(ctx.h, ts[i]):
                left.discard(i)
        if not left:
            break
    assert not left
    for q, a in zip(qs, alone):
        assert np.array_equal(q["out"], oracle_out(paper_keys, q))
        assert np.array_equal(q["out"], a)
    ctx.close()


def test_submit_errors():
    ctx, s = gpu_ctx()
    bad = vp.Query(7, 0, 0, 0, None, None, None, None, 1, None)
    with pytest.raises(vp.VelopirError):
        vp.velopir_submit(ctx.h, bad)
    with pytest.raises(vp.VelopirError):
        vp.velopir_poll(ctx.h, 10 ** 9)


def test_progress_reports_every_ticket_once(paper_keys):
    """velopir_progress steps the loop and reports each finished ticket once;
    results equal the queries run alone."""
    ctx, s = gpu_ctx()
    qs = make_queries(s, 4, fanin=4)
    alone = [run_alone(ctx, q) for q in qs]
    tickets = {vp.velopir_submit(ctx.h, as_record(q)): i for i, q in enumerate(qs)}
    seen = []
    for _ in range(500):
        seen += vp.velopir_progress(ctx.h)
        if len(seen) == len(qs):
            break
    assert sorted(seen) == sorted(tickets)
    assert vp.velopir_progress(ctx.h) == []
    for q, a in zip(qs, alone):
        assert np.array_equal(q["out"], oracle_out(paper_keys, q))
        assert np.array_equal(q["out"], a)


def test_cancel_waiting_and_admitted_queries(paper_keys):
    """A query cancelled before admission, or while its layers run, is
    reported once as cancelled (velopir_poll raises ERR_CANCELLED); the others
    finish with the results they have alone, and admitted memory is released."""
    ctx, s = gpu_ctx()
    qs = make_queries(s, 3)            # IntV (34 layers), CoV, IdM
    alone = [run_alone(ctx, q) for q in qs]
    ts = [vp.velopir_submit(ctx.h, as_record(q)) for q in qs]
    vp.velopir_cancel(ctx.h, ts[1])    # still waiting: dropped at once
    with pytest.raises(vp.VelopirError) as e:
        vp.velopir_poll(ctx.h, ts[1])
    assert e.value.code == vp.ERRORS_BY_NAME["ERR_CANCELLED"]
    assert vp.velopir_poll(ctx.h, ts[0]) is False   # admits the rest, issues one step
    vp.velopir_cancel(ctx.h, ts[0])    # admitted, most layers still to go
    done, cancelled = set(), set()
    for _ in range(500):
        for i in (0, 2):
            if i in done or i in cancelled:
                continue
            try:
                if vp.velopir_poll(ctx.h, ts[i]):
                    done.add(i)
            except vp.VelopirError as err:
                assert err.code == vp.ERRORS_BY_NAME["ERR_CANCELLED"]
                cancelled.add(i)
        if len(done) + len(cancelled) == 2:
            break
    assert cancelled == {0} and done == {2}
    assert np.array_equal(qs[2]["out"], oracle_out(paper_keys, qs[2]))
    assert np.array_equal(qs[2]["out"], alone[2])
    assert vp.velopir_queue_depth(ctx.h) == (0, 0)
    with pytest.raises(vp.VelopirError):
        vp.velopir_cancel(ctx.h, 10 ** 9)


def test_issue_thread_serves_staggered_arrivals(paper_keys):
    """With the library's issue thread running, queries submitted while
    others are on the GPU finish without the caller stepping the loop; every
    result equals the oracle's, and non-serving calls are refused until the
    thread stops."""
    import time
    ctx, s = gpu_ctx()
    qs = make_queries(s, 3) + make_queries(s, 4, fanin=4)
    vp.velopir_serve_start(ctx.h)
    try:
        with pytest.raises(vp.VelopirError) as e:
            vp.velopir_sync(ctx.h)
        assert e.value.code == vp.ERRORS_BY_NAME["ERR_BUSY"]
        tickets = {}
        for i, q in enumerate(qs):
            tickets[vp.velopir_submit(ctx.h, as_record(q))] = i
            time.sleep(0.05)
        seen = set()
        t0 = time.time()
        while len(seen) < len(qs):
            seen.update(vp.velopir_progress(ctx.h))
            time.sleep(0.01)
            assert time.time() - t0 < 300
        assert seen == set(tickets)
    finally:
        vp.velopir_serve_stop(ctx.h)
    vp.velopir_sync(ctx.h)
    for q in qs:
        assert np.array_equal(q["out"], oracle_out(paper_keys, q))
    assert vp.velopir_queue_depth(ctx.h) == (0, 0)


def test_serving_mix_traced_at_scale(paper_keys):
    """The serving workload's 40/30/30 IntV/CoV/IdM mix at sizes a test can
    afford (IntV D = 256 and 128; CoV D = 1,024 and 512; IdM-32 D = 2,048
    and 1,024 with payloads aggregated by fan-in 8: 207,232 bootstraps),
    arriving one every few serving steps while the others run.  Of every
    serving step's launches a seeded sample of >= 4,096 gates in all is
    recomputed by the oracle from the recorded inputs (bit-identical), and
    every output decrypts to its plaintext answer."""
    ctx, s = gpu_ctx()
    vp.velopir_set_path(ctx.h, vp.VP_PATH_NTT)
    qs, answers = [], []
    for k, D in enumerate((256, 128)):
        w = synth.intv_workload(D, substream=60 + k)
        cx = encrypt_value_bits(s, w["x"], 32, 960 + 2 * k)
        cy = encrypt_value_bits(s, w["y"], 32, 961 + 2 * k)
        r = np.ascontiguousarray(w["rects"], dtype=np.uint32)
        qs.append(dict(kind=vp.VP_QUERY_INTV, a=cx, b=cy, db=r, D=D, out=np.zeros((D, 631), np.uint32)))
        r64 = r.astype(np.int64)
        answers.append(((r64[:, 0] <= w["x"]) & (w["x"] < r64[:, 1]) & (r64[:, 2] <= w["y"]) &
                        (w["y"] < r64[:, 3])).astype(np.uint32))
    for k, D in enumerate((1024, 512)):
        w = synth.cov_workload(D, substream=62 + k)
        cell = encrypt_value_bits(s, w["cell"], 32, 964 + k)
        cells = w["cells"].astype(np.uint32)
        qs.append(dict(kind=vp.VP_QUERY_COV, a=cell, db=cells, D=D, out=np.zeros((D, 631), np.uint32)))
        answers.append((cells == w["cell"]).astype(np.uint32))
    for k, D in enumerate((2048, 1024)):
        w = synth.idm_workload(D, 32, distinct=True, payload=True, substream=64 + k)
        x = encrypt_value_bits(s, w["query"], 32, 966 + k)
        pay = w["payload"].astype(np.uint32)
        qs.append(dict(kind=vp.VP_QUERY_IDM, a=x, db=w["ids"].astype(np.uint32), D=D, id_bits=32, payload=pay,
                       payload_bits=32, out=np.zeros((32, 631), np.uint32), fanin=8))
        answers.append(np.array([(int(pay[w["planted"]]) >> j) & 1 for j in range(32)], dtype=np.uint32))
    vp.velopir_trace_start(ctx.h, 35, 16, 48, 8192)      # >= 207,232 / 48 = 4,318 gates
    order = [0, 2, 4, 1, 3, 5]          # arrivals alternate between the modes
    tickets, seen, steps, nxt = {}, set(), 0, 0
    while len(seen) < len(qs):
        if nxt < len(order) and steps % 3 == 0:
            tickets[vp.velopir_submit(ctx.h, as_record(qs[order[nxt]]))] = order[nxt]
            nxt += 1
        seen.update(vp.velopir_progress(ctx.h))
        steps += 1
        assert steps < 5000
    recs = vp.velopir_trace_stop(ctx.h, 8192)
    assert seen == set(tickets) and vp.velopir_queue_depth(ctx.h) == (0, 0)
    assert len(recs) < 8192, "the trace buffer filled up: later steps were not sampled"
    for q, want in zip(qs, answers):
        assert np.array_equal(vp.velopir_client_decrypt_bits(s, q["out"]), want), q["kind"]
    check_trace(paper_keys, recs, 4096)
