"""Serving benchmark: mixed-mode queries with Poisson arrivals through the
continuous-batching loop (velopir_submit / velopir_progress), with the
library's issue thread stepping the loop (velopir_serve_start) so the GPU
does not wait for the caller.

Mix (shaped like the paper's three modes): 40% interval validation with D
log-uniform in [256, 4096], 30% coordinate validation with D in [256, 16384],
30% identifier matching (32-bit ids, 32-bit payload aggregation, fan-in
--fanin) with D in [1024, 65536].  Capacity is measured closed-loop (all
queries submitted at once); then each load point replays Poisson arrivals at
a multiple of that capacity and reports query latency p50/p99 (arrival to
completion) over its queries after the first --warmup of the point, with the
achieved against the offered rate.

    python -m paper_2506_12761_gb300.serve_bench --per-point 60 --loads 0.25,0.5,0.75,1.0,1.25,1.5
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, synth
from . import velopir as vp


def fanin_nodes(D: int, g: int) -> int:
    """Bootstraps per payload bit of the XOR aggregation tree of fan-in g."""
    nodes, k = 0, 1
    while k < D:
        nodes += sum(1 for i in range(0, D, g * k) if sum(1 for m in range(g) if i + m * k < D) >= 2)
        k *= g
    return nodes


def query_shape(q: int, seed: int):
    """Mode and database size of query q of the mix (the draws make_query uses)."""
    st = synth.Stream(seed, synth.STREAM_ARRIVALS, 1000 + q)
    u = float(st.unit_doubles(1)[0])
    kind = 0 if u < 0.4 else (1 if u < 0.7 else 2)
    lo, hi = [(256, 4096), (256, 16384), (1024, 65536)][kind]
    return kind, int(synth.log_uniform_sizes(1, lo, hi, seed=seed, substream=2000 + q)[0])


def bootstraps_of(kind: int, D: int, fanin: int) -> int:
    if kind == 0:
        return 131 * D
    if kind == 1:
        return 31 * D
    return 31 * D + 32 * fanin_nodes(D, fanin)


def mix_mean_bootstraps(seed: int, fanin: int, n: int = 2000, first: int = 100000) -> float:
    """Mean bootstraps per query of the mix, over n queries of the same
    generator (sizes only, nothing runs): the capacity in queries/s is the
    measured bootstraps/s divided by it."""
    return float(np.mean([bootstraps_of(*query_shape(first + q, seed), fanin) for q in range(n)]))


def make_query(s, q: int, seed: int, fanin: int = 2):
    kind, D = query_shape(q, seed)
    if kind == 0:
        w = synth.intv_workload(D, seed=seed, substream=3000 + q)
        a = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["x"]], 32)[0], synth.lwe_material(32, seed=seed, substream=4000 + 2 * q))
        b = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["y"]], 32)[0], synth.lwe_material(32, seed=seed, substream=4001 + 2 * q))
        r = w["rects"].astype(np.int64)
        want = ((r[:, 0] <= w["x"]) & (w["x"] < r[:, 1]) & (r[:, 2] <= w["y"]) & (w["y"] < r[:, 3])).astype(np.uint32)
        return dict(kind=vp.VP_QUERY_INTV, a=a, b=b, db=np.ascontiguousarray(w["rects"], dtype=np.uint32), D=D,
                    out=np.zeros((D, 631), np.uint32), want=want, boots=131 * D)
    if kind == 1:
        w = synth.cov_workload(D, seed=seed, substream=3000 + q)
        a = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["cell"]], 32)[0], synth.lwe_material(32, seed=seed, substream=4000 + 2 * q))
        cells = w["cells"].astype(np.uint32)
        return dict(kind=vp.VP_QUERY_COV, a=a, db=cells, D=D, out=np.zeros((D, 631), np.uint32),
                    want=(cells == w["cell"]).astype(np.uint32), boots=31 * D)
    w = synth.idm_workload(D, 32, seed=seed, substream=3000 + q, distinct=True, payload=True)
    a = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["query"]], 32)[0], synth.lwe_material(32, seed=seed, substream=4000 + 2 * q))
    pay = w["payload"].astype(np.uint32)
    return dict(kind=vp.VP_QUERY_IDM, a=a, db=w["ids"].astype(np.uint32), D=D, id_bits=32, payload=pay,
                payload_bits=32, out=np.zeros((32, 631), np.uint32), fanin=fanin,
                want=synth.value_bits([int(pay[w["planted"]])], 32)[0], boots=31 * D + 32 * fanin_nodes(D, fanin))


def record(q):
    return vp.make_query(q["kind"], q["a"], q["db"], q["D"], q["out"], enc_b=q.get("b"), id_bits=q.get("id_bits", 0),
                         payload=q.get("payload"), payload_bits=q.get("payload_bits", 0),
                         agg_fanin=q.get("fanin", 0))


def run(ctx, queries, arrivals, threaded: bool):
    """Submit each query at its arrival time (seconds from start).  With the
    issue thread the caller only submits and collects; otherwise it steps the
    loop itself whenever work is in flight.  Returns per-query completion
    times (s from start) and the wall time."""
    n = len(queries)
    recs = [record(q) for q in queries]
    t0 = time.perf_counter()
    nxt, ticket_of, done_at = 0, {}, {}
    while len(done_at) < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            ticket_of[vp.velopir_submit(ctx, recs[nxt])] = nxt
            nxt += 1
        if threaded:
            for t in vp.velopir_progress(ctx):
                done_at[ticket_of[t]] = time.perf_counter() - t0
            time.sleep(0.002 if nxt >= n else max(0.0, min(0.002, arrivals[nxt] - now)))
            continue
        adm, wait = vp.velopir_queue_depth(ctx)
        if adm or wait:
            for t in vp.velopir_progress(ctx):
                done_at[ticket_of[t]] = time.perf_counter() - t0
        elif nxt < n:
            time.sleep(max(0.0, min(0.05, arrivals[nxt] - now)))
    wall = time.perf_counter() - t0
    return np.array([done_at[i] for i in range(n)]), wall


def check(s, queries):
    ok = 0
    for q in queries:
        bits = vp.velopir_client_decrypt_bits(s, q["out"])
        ok += int(np.array_equal(bits, q["want"]))
    return ok


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--per-point", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=0, help="queries at the start of each point left out of p50/p99")
    ap.add_argument("--capacity-queries", type=int, default=8)
    ap.add_argument("--loads", default="0.5,1.0,1.5")
    ap.add_argument("--budget-gb", type=float, default=96.0)
    ap.add_argument("--fanin", type=int, default=8, help="IdM aggregation fan-in (2: the pairwise HomSum)")
    ap.add_argument("--no-thread", action="store_true", help="step the loop from the caller (no issue thread)")
    ap.add_argument("--seed", type=int, default=synth.MASTER_SEED)
    args = ap.parse_args()
    build.build()
    km = synth.key_material(args.seed)
    bk, ksk = vp.velopir_client_keygen(km)
    ctx = vp.Context(0, int(args.budget_gb * (1 << 30)))
    vp.velopir_load_cloud_key(ctx.h, bk, ksk)
    vp.velopir_autotune(ctx.h)
    threaded = not args.no_thread
    if threaded:
        vp.velopir_serve_start(ctx.h)
    # closed loop: every query at t = 0, for the sustained bootstraps/s; the
    # capacity in queries/s is that rate over the mix's mean query size (a
    # dozen queries are too few to estimate the mean of sizes spread over
    # more than two orders of magnitude)
    cap_q = [make_query(km.s, q, args.seed, args.fanin) for q in range(args.capacity_queries)]
    done, wall = run(ctx.h, cap_q, np.zeros(len(cap_q)), threaded)
    boots = sum(q["boots"] for q in cap_q)
    mean_boots = mix_mean_bootstraps(args.seed, args.fanin)
    capacity = boots / wall / mean_boots
    result = {"metric": "query latency p50/p99 (ms) and throughput under Poisson load, mixed IntV/CoV/IdM",
              "issue_thread": threaded, "idm_aggregation_fanin": args.fanin,
              "capacity": {"queries_per_s": capacity, "bootstraps_per_s": boots / wall, "queries": len(cap_q),
                           "seconds": wall, "mean_bootstraps_per_query": mean_boots,
                           "correct": check(km.s, cap_q)},
              "points": []}
    print(json.dumps(result["capacity"]), flush=True)
    base = args.capacity_queries
    for li, load in enumerate(float(x) for x in args.loads.split(",")):
        qs = [make_query(km.s, base + q, args.seed, args.fanin) for q in range(args.per_point)]
        base += args.per_point
        arr = synth.poisson_arrivals(len(qs), load * capacity, seed=args.seed, substream=li)
        arr = arr - arr[0]
        done, wall = run(ctx.h, qs, arr, threaded)
        lat = done - arr
        k = min(args.warmup, len(qs) - 1)
        span = float(done[k:].max() - arr[k])          # first counted arrival to last completion
        kinds = {0: "intv", 1: "cov", 2: "idm"}
        per_mode = {kinds[m]: float(np.percentile(lat[k:][[q["kind"] == m for q in qs[k:]]], 50) * 1e3)
                    for m in kinds if any(q["kind"] == m for q in qs[k:])}
        result["points"].append({"offered_load": load, "offered_qps": load * capacity,
                                 "queries": len(qs), "counted": len(qs) - k,
                                 "p50_ms": float(np.percentile(lat[k:], 50) * 1e3),
                                 "p99_ms": float(np.percentile(lat[k:], 99) * 1e3),
                                 "p50_ms_by_mode": per_mode,
                                 "achieved_qps": (len(qs) - k) / span,
                                 "bootstraps_per_s": sum(q["boots"] for q in qs[k:]) / span,
                                 "correct": check(km.s, qs)})
        print(json.dumps(result["points"][-1]), flush=True)
    if threaded:
        vp.velopir_serve_stop(ctx.h)
    print(json.dumps(result), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
