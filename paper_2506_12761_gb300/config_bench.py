"""Timed runs of the workloads beside the benchmark's interval query, each
checked by decrypting every output against its plaintext answer:

  idm8     identifier matching, 8-bit id, D = 4 (7-AND tree per entry, 28 bootstraps)
  idm32    identifier matching, 32-bit id, D = 65,536 distinct ids: match bits
           (31-AND tree per entry, 2,031,616 bootstraps), then the same query
           with each entry's 32-bit payload zeroed by its match bit and
           XOR-aggregated: pairwise (Section 5's HomSum, + 2,097,120
           bootstraps) and with fan-in 4 and 8 (one bootstrap per 4 or 8
           inputs, + 32 x 21,845 and + 32 x 9,363)
  cov64    64 coordinate queries (16+16-bit cells), D log-uniform in
           [256, 16384], one program captured in a CUDA graph

  intv_encdb  interval validation over an encrypted database (Alg. ServerEnc
              ciphertexts), l_I = 16, D = 1,024: 195 bootstraps per entry
  paper4   the paper's full protocol (encrypted database, validation,
           HomBitwiseAND with the encrypted payload, HomSum aggregation) on
           synthetic stand-ins with the shapes of its Table 4 datasets
           (M entries, l_I = 16, payload l_S bits): covid-kor IntV/IdM
           (M = 9, l_S = 9), covid-usa IntV/IdM (58, 22), gdacs CoV (9, 16),
           weather-usa IdM (304, 128); printed beside the paper's "All"
           times, which were measured on its CPU + RTX 4060 Ti (context only)
  client   the client-side preprocessing on the GPU (velopir_gpu_keygen,
           velopir_gpu_pubkeygen; device buffers) beside the host client
           library on the machine's cores: the cloud key (BK 31 MB, KSK 83 MB) and
           32,768 encryptions of zero (Alg. PubKeyGen), outputs compared

Inputs are synthetic and seeded (synth).  Times are wall-clock around the
synchronous library calls (host buffers in and out, program scheduling
included), after the tile-shape autotuner.

    python -m paper_2506_12761_gb300.config_bench --which idm8,idm32,cov64,intv_encdb,paper4
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


def fanin_nodes(D: int, g: int) -> int:
    """Bootstraps per payload bit of the XOR aggregation tree of fan-in g."""
    nodes, k = 0, 1
    while k < D:
        nodes += sum(1 for i in range(0, D, g * k) if sum(1 for m in range(g) if i + m * k < D) >= 2)
        k *= g
    return nodes


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
    rows = [{"workload": "idm32 D=65536 match bits", "bootstraps": b_match, "seconds": t_match,
             "bootstraps_per_s": b_match / t_match, "correct": bool(ok_match)},
            {"workload": "idm32 D=65536 payload XOR aggregation (pairwise HomSum)", "bootstraps": b_agg,
             "seconds": t_agg, "bootstraps_per_s": b_agg / t_agg, "correct": bool(ok_agg)}]
    for g in (4, 8):   # the cheaper aggregation: one bootstrap per g inputs
        agg = np.zeros((32, 631), dtype=np.uint32)
        t0 = time.perf_counter()
        vp.velopir_query_batch(ctx, [vp.make_query(vp.VP_QUERY_IDM, x, ids, D, agg, id_bits=32, payload=pay,
                                                   payload_bits=32, agg_fanin=g)])
        t_g = time.perf_counter() - t0
        got = vp.velopir_client_decrypt_bits(s, agg)
        ok_g = sum(int(b) << j for j, b in enumerate(got)) == int(pay[w["planted"]])
        b_g = 31 * D + 32 * fanin_nodes(D, g)
        rows.append({"workload": f"idm32 D=65536 payload XOR aggregation, fan-in {g}", "bootstraps": b_g,
                     "seconds": t_g, "bootstraps_per_s": b_g / t_g, "correct": bool(ok_g)})
    return rows


def run_cov64(ctx, s):
    sizes = synth.log_uniform_sizes(64, 256, 16384, substream=9)
    recs, checks, keep = [], [], []   # the records hold raw pointers: keep every buffer alive
    for q, D in enumerate(sizes):
        w = synth.cov_workload(int(D), substream=100 + q)
        cell = vp.velopir_client_encrypt_bits(s, synth.value_bits([w["cell"]], 32)[0],
                                              synth.lwe_material(32, substream=200 + q))
        cells = w["cells"].astype(np.uint32)
        out = np.zeros((int(D), 631), dtype=np.uint32)
        recs.append(vp.make_query(vp.VP_QUERY_COV, cell, cells, int(D), out))
        keep.append((cell, cells))
        checks.append((out, (cells == w["cell"]).astype(np.uint32)))
    t0 = time.perf_counter()
    vp.velopir_query_batch(ctx, recs, use_graph=True)
    dt = time.perf_counter() - t0
    ok = all(np.array_equal(vp.velopir_client_decrypt_bits(s, o), want) for o, want in checks)
    boots = int(31 * np.sum(sizes))
    return {"workload": "cov64: 64 queries, D log-uniform [256,16384], one graph", "queries": 64,
            "total_D": int(np.sum(sizes)), "bootstraps": boots, "seconds": dt, "bootstraps_per_s": boots / dt,
            "correct": bool(ok)}


def server_enc(s, values, width, seed):
    """Alg. PubKeyGen + ServerEnc of plaintext values: [len(values)][width][631]."""
    bits = synth.value_bits(np.asarray(values, dtype=np.uint64), width)
    pk = vp.velopir_client_pubkeygen(s, synth.lwe_material(bits.size, seed=seed, stream=synth.STREAM_PUBKEY))
    return vp.velopir_server_encrypt(pk, bits.reshape(-1)).reshape(len(values), width, 631)


def intv_case(M, l, sub):
    """A 16-bit point and M rectangles, every third containing it."""
    st = synth.Stream(synth.MASTER_SEED, synth.STREAM_DB, sub)
    mask = (1 << l) - 1
    x, y = (int(v) & mask for v in st.words(2))
    u = (st.words(4 * M) & np.uint32(mask)).reshape(M, 4).astype(np.int64)
    lo, hi = np.minimum(u[:, [0, 2]], u[:, [1, 3]]), np.maximum(u[:, [0, 2]], u[:, [1, 3]]) + 1
    lo[::3, 0], hi[::3, 0], lo[::3, 1], hi[::3, 1] = max(0, x - 7), x + 1, y, y + 9
    hi = np.minimum(hi, mask)
    rects = np.stack([lo[:, 0], hi[:, 0], lo[:, 1], hi[:, 1]], axis=1).astype(np.uint32)
    r = rects.astype(np.int64)
    valid = ((r[:, 0] <= x) & (x < r[:, 1]) & (r[:, 2] <= y) & (y < r[:, 3])).astype(np.uint32)
    return x, y, rects, valid


def run_intv_encdb(ctx, s):
    D, l = 1024, 16
    x, y, rects, valid = intv_case(D, l, 40)
    cx = vp.velopir_client_encrypt_bits(s, synth.value_bits([x], l)[0], synth.lwe_material(l, substream=41))
    cy = vp.velopir_client_encrypt_bits(s, synth.value_bits([y], l)[0], synth.lwe_material(l, substream=42))
    enc = server_enc(s, rects.reshape(-1), l, 43)
    out = np.zeros((D, 631), dtype=np.uint32)
    t0 = time.perf_counter()
    vp.velopir_interval_query_encdb(ctx, cx, cy, l, enc, D, None, 0, out)
    dt = time.perf_counter() - t0
    ok = np.array_equal(vp.velopir_client_decrypt_bits(s, out), valid)
    boots = (12 * l + 3) * D
    return {"workload": "intv_encdb: encrypted database, l_I=16, D=1024", "bootstraps": boots, "seconds": dt,
            "bootstraps_per_s": boots / dt, "correct": bool(ok)}


PAPER4 = [  # dataset, mode, M, l_S, the paper's "All" time (s), Table 4
    ("covid-kor", "IntV", 9, 9, 2.512), ("covid-kor", "IdM", 9, 9, 1.13875),
    ("covid-usa", "IntV", 58, 22, 9.82627), ("covid-usa", "IdM", 58, 22, 7.95777),
    ("gdacs", "CoV", 9, 16, 1.12841), ("weather-usa", "IdM", 304, 128, 65.7115),
]


def paper4_case(s, k: int) -> dict:
    """The inputs of Table 4 shape k (PAPER4): an encrypted database of M
    entries with l_I = 16-bit values, an encrypted l_S-bit payload per entry
    (Alg. PubKeyGen + ServerEnc), the encrypted query, and the plaintext
    answer (the XOR of the payloads of the valid entries)."""
    l = 16
    name, mode, M, lS, paper_s = PAPER4[k]
    st = synth.Stream(synth.MASTER_SEED, synth.STREAM_DB, 60 + k)
    pay = (st.words(M) & np.uint32((1 << min(lS, 32)) - 1)).astype(np.uint64)
    pay_bits = synth.value_bits(pay, 32)[:, :lS] if lS <= 32 else st.bits(M * lS).reshape(M, lS).astype(np.uint32)
    P = vp.velopir_server_encrypt(
        vp.velopir_client_pubkeygen(s, synth.lwe_material(M * lS, seed=70 + k, stream=synth.STREAM_PUBKEY)),
        pay_bits.reshape(-1)).reshape(M, lS, 631)
    c = dict(name=name, mode=mode, M=M, lS=lS, l=l, paper_s=paper_s, P=P)
    if mode == "IntV":
        x, y, rects, valid = intv_case(M, l, 80 + k)
        c.update(cx=vp.velopir_client_encrypt_bits(s, synth.value_bits([x], l)[0], synth.lwe_material(l, substream=90 + k)),
                 cy=vp.velopir_client_encrypt_bits(s, synth.value_bits([y], l)[0], synth.lwe_material(l, substream=100 + k)),
                 enc=server_enc(s, rects.reshape(-1), l, 110 + k), valid=valid, boots=(12 * l + 3) * M)
    elif mode == "CoV":
        cells = st.words(M)
        valid = np.zeros(M, dtype=np.uint32)
        valid[M // 2] = 1
        q = int(cells[M // 2])
        c.update(cq=vp.velopir_client_encrypt_bits(s, synth.value_bits([q], 2 * l)[0],
                                                   synth.lwe_material(2 * l, substream=90 + k)),
                 enc=server_enc(s, cells, 2 * l, 110 + k), valid=valid, boots=(4 * l - 1) * M)
    else:
        ids = synth.distinct_u32(st, M, l).astype(np.uint32)
        valid = np.zeros(M, dtype=np.uint32)
        valid[M // 3] = 1
        c.update(xq=vp.velopir_client_encrypt_bits(s, synth.value_bits([int(ids[M // 3])], l)[0],
                                                   synth.lwe_material(l, substream=90 + k)),
                 enc=server_enc(s, ids, l, 110 + k), valid=valid, boots=(2 * l - 1) * M)
    c["boots"] += M * lS + (M - 1) * lS   # HomBitwiseAND + HomSum
    want = np.zeros(lS, dtype=np.uint32)
    for d in np.flatnonzero(c["valid"]):
        want ^= pay_bits[d].astype(np.uint32)
    c["want"] = want
    return c


def paper4_run(ctx, c, out) -> None:
    """Run the full protocol of a paper4_case through the C ABI into out [l_S][631]."""
    if c["mode"] == "IntV":
        vp.velopir_interval_query_encdb(ctx, c["cx"], c["cy"], c["l"], c["enc"], c["M"], c["P"], c["lS"], out)
    elif c["mode"] == "CoV":
        vp.velopir_coordinate_query_encdb(ctx, c["cq"], c["l"], c["enc"], c["M"], c["P"], c["lS"], out)
    else:
        vp.velopir_id_match_encdb(ctx, c["xq"], c["l"], c["enc"], c["M"], c["P"], c["lS"], out)


def run_paper4(ctx, s):
    """Each Table 4 shape with Section 5's pairwise HomSum, then with the
    fan-in-8 XOR tree (velopir_set_encdb_fanin)."""
    res = []
    for k in range(len(PAPER4)):
        c = paper4_case(s, k)
        for g in (2, 8):
            boots = c["boots"] - (c["M"] - 1) * c["lS"] + fanin_nodes(c["M"], g) * c["lS"]
            out = np.zeros((c["lS"], 631), dtype=np.uint32)
            vp.velopir_set_encdb_fanin(ctx, g)
            t0 = time.perf_counter()
            paper4_run(ctx, c, out)
            dt = time.perf_counter() - t0
            vp.velopir_set_encdb_fanin(ctx, 0)
            ok = np.array_equal(vp.velopir_client_decrypt_bits(s, out), c["want"])
            agg = "pairwise HomSum" if g == 2 else f"fan-in {g} XOR tree"
            res.append({"workload": f"paper4 {c['name']} {c['mode']} (encrypted database, M={c['M']}, "
                                    f"l_I={c['l']}, l_S={c['lS']}, {agg})",
                        "bootstraps": boots, "seconds": dt, "bootstraps_per_s": boots / dt,
                        "paper_all_seconds": c["paper_s"], "correct": bool(ok)})
    return res


def run_client(ctx, s):
    """Cloud key and Alg. PubKeyGen on the GPU against the host client library."""
    import torch

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()

    km = synth.key_material()
    t0 = time.perf_counter()
    bk_h, ksk_h = vp.velopir_client_keygen(km)
    t_host = time.perf_counter() - t0
    dkm = type("Km", (), {k: dev(getattr(km, k)) for k in ("s", "K", "bk_a", "bk_e", "ksk_a", "ksk_e")})
    bk = torch.zeros(vp.BK_WORDS, dtype=torch.int32, device="cuda")
    ksk = torch.zeros(vp.KSK_WORDS, dtype=torch.int32, device="cuda")
    vp.velopir_gpu_keygen(ctx, dkm, bk, ksk)        # warm
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        vp.velopir_gpu_keygen(ctx, dkm, bk, ksk)
        ts.append(time.perf_counter() - t0)
    same = bool(np.array_equal(bk.cpu().numpy().view(np.uint32), bk_h) and
                np.array_equal(ksk.cpu().numpy().view(np.uint32), ksk_h))
    res = [{"workload": "cloud key (BK + KSK)", "host_client_s": t_host, "gpu_s": float(min(ts)),
            "speedup": t_host / min(ts), "correct": same}]
    # 32,768 encryptions of zero, with the key-switching key's masks and noises as material
    a = np.ascontiguousarray(km.ksk_a.reshape(-1, 630), dtype=np.uint32)
    e = np.ascontiguousarray(km.ksk_e.reshape(-1), dtype=np.uint32)
    lm = synth.LweMaterial(a, e)
    t0 = time.perf_counter()
    pk_h = vp.velopir_client_pubkeygen(s, lm)
    t_host = time.perf_counter() - t0
    da, de, ds = dev(a), dev(e), dev(s)
    pk = torch.zeros((e.size, 631), dtype=torch.int32, device="cuda")
    vp.velopir_gpu_pubkeygen(ctx, ds, da, de, pk)   # warm
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        vp.velopir_gpu_pubkeygen(ctx, ds, da, de, pk)
        ts.append(time.perf_counter() - t0)
    res.append({"workload": f"Alg. PubKeyGen, {e.size} encryptions of zero", "host_client_s": t_host,
                "gpu_s": float(min(ts)), "speedup": t_host / min(ts),
                "correct": bool(np.array_equal(pk.cpu().numpy().view(np.uint32), pk_h))})
    return res


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
    runs = {"idm8": run_idm8, "idm32": run_idm32, "cov64": run_cov64, "intv_encdb": run_intv_encdb,
            "paper4": run_paper4, "client": run_client}
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
