"""Timed runs of the workloads beside the benchmark's interval query, each
checked by decrypting every output against its plaintext answer:

  idm8     identifier matching, 8-bit id, D = 4 (7-AND tree per entry, 28 bootstraps)
  idm32    identifier matching, 32-bit id, D = 65,536 distinct ids: match bits
           (31-AND tree per entry, 2,031,616 bootstraps), then the same query
           with each entry's 32-bit payload zeroed by its match bit and
           XOR-aggregated (HomSum, + 2,097,120 bootstraps)
  cov64    64 coordinate queries (16+16-bit cells), D log-uniform in
           [256, 16384], one program captured in a CUDA graph

Inputs are synthetic and seeded (synth).  Times are wall-clock around the
synchronous library calls (host buffers in and out, program scheduling
included), after the tile-shape autotuner.

    python -m paper_2506_12761_gb300.config_bench --which idm8,idm32,cov64
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, synth
from . import velopir as vp


def run_idm8(ctx, s):
    D = 4
    w = synth.idm_workload(D, 8, distinct=True)
    x = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["query"]], 8)[0], synth.lwe_material(8, substream=31))
    ids = w["ids"].astype(np.uint32)
    out = np.zeros((D, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx, x, 8, ids, D, None, 0, out)   # warm
    t0 = time.perf_counter()
    vp.velopir_id_match(ctx, x, 8, ids, D, None, 0, out)
    dt = time.perf_counter() - t0
    ok = np.array_equal(vp.velopir_client_decrypt_bits(s, out), (ids == w["query"]).astype(np.uint32))
    return {"workload": "idm8 D=4", "bootstraps": 7 * D, "seconds": dt, "query_ms": dt * 1e3, "correct": bool(ok)}


def run_idm32(ctx, s):
    D = 65536
    w = synth.idm_workload(D, 32, distinct=True, payload=True)
    x = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["query"]], 32)[0], synth.lwe_material(32, substream=5))
    ids = w["ids"].astype(np.uint32)
    pay = w["payload"].astype(np.uint32)
    match = np.zeros((D, 631), dtype=np.uint32)
    t0 = time.perf_counter()
    vp.velopir_id_match(ctx, x, 32, ids, D, None, 0, match)
    t_match = time.perf_counter() - t0
    bits = vp.velopir_client_decrypt_bits(s, match)
    ok_match = int(bits.sum()) == 1 and int(bits[w["planted"]]) == 1
    agg = np.zeros((32, 631), dtype=np.uint32)
    t0 = time.perf_counter()
    vp.velopir_id_match(ctx, x, 32, ids, D, pay, 32, agg)
    t_agg = time.perf_counter() - t0
    got = vp.velopir_client_decrypt_bits(s, agg)
    ok_agg = sum(int(b) << j for j, b in enumerate(got)) == int(pay[w["planted"]])
    b_match = 31 * D
    b_agg = 31 * D + 32 * (D - 1)
    return [{"workload": "idm32 D=65536 match bits", "bootstraps": b_match, "seconds": t_match,
             "bootstraps_per_s": b_match / t_match, "correct": bool(ok_match)},
            {"workload": "idm32 D=65536 payload XOR aggregation", "bootstraps": b_agg, "seconds": t_agg,
             "bootstraps_per_s": b_agg / t_agg, "correct": bool(ok_agg)}]


def run_cov64(ctx, s):
    sizes = synth.log_uniform_sizes(64, 256, 16384, substream=9)
    recs, checks = [], []
    for q, D in enumerate(sizes):
        w = synth.cov_workload(int(D), substream=100 + q)
        cell = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["cell"]], 32)[0],
                                              synth.lwe_material(32, substream=200 + q))
        cells = w["cells"].astype(np.uint32)
        out = np.zeros((int(D), 631), dtype=np.uint32)
        recs.append(vp.make_query(vp.VP_QUERY_COV, cell, cells, int(D), out))
        checks.append((out, (cells == w["cell"]).astype(np.uint32)))
    t0 = time.perf_counter()
    vp.velopir_query_batch(ctx, recs, use_graph=True)
    dt = time.perf_counter() - t0
    ok = all(np.array_equal(vp.velopir_client_decrypt_bits(s, o), want) for o, want in checks)
    boots = int(31 * np.sum(sizes))
    return {"workload": "cov64: 64 queries, D log-uniform [256,16384], one graph", "queries": 64,
            "total_D": int(np.sum(sizes)), "bootstraps": boots, "seconds": dt, "bootstraps_per_s": boots / dt,
            "correct": bool(ok)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--which", default="idm8,idm32,cov64")
    args = ap.parse_args()
    build.build()
    km = synth.key_material()
    bk, ksk = vp.velopir_client_keygen(km)
    ctx = vp.Context(0)
    vp.velopir_load_cloud_key(ctx.h, bk, ksk)
    vp.velopir_autotune(ctx.h)
    runs = {"idm8": run_idm8, "idm32": run_idm32, "cov64": run_cov64}
    ok = True
    for name in args.which.split(","):
        res = runs[name](ctx.h, km.s)
        for r in (res if isinstance(res, list) else [res]):
            ok &= r["correct"]
            print(json.dumps(r), flush=True)
    ctx.close()
    if not ok:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
