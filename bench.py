"""Benchmark: gate bootstraps/s of batched TFHE gate bootstrapping on GB300.

One step = one interval-validation query (Alg. InterValid) over D = 1,024
plaintext rectangles with a 32-bit unsigned encrypted point: 131 bootstraps
per entry, 134,144 per step: 34 gate layers, list-scheduled into launches
of whole waves of the blind-rotation kernel.  Inputs and keys
are synthetic and seeded (paper_2506_12761_gb300.synth), shaped like the
paper's interval-validation workload.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
only reference implementation this project has) on a bounded sample of the
same workload.  Under torchrun each rank runs its own replica of the query
(weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gate bootstraps/sec on 1 GB300 (n=630,N=1024) batched vs plain; query p50/p99 ms"
UNIT = "bootstraps/s"
D = 1024
BOOTSTRAPS_PER_STEP = 131 * D
WORKLOAD = ("interval validation: 32-bit unsigned encrypted point vs D=1024 plaintext rectangles, "
            "131 bootstraps/entry = 134,144 bootstraps/step (34 gate layers, list-scheduled into launches of "
            "whole waves); TFHE n=630 N=1024 l=3 Bg=2^7 t=8")
MACS_DENSE = 12 * 1024 * 1024 * 630          # int32 multiply-adds per bootstrap, dense contraction


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class Dist:
    def __init__(self, world):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p:
            self.p.terminate()
            self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def traffic_for(kernel_src: str):
    """DRAM bytes per launch (read + write) of the dominant kernel from the
    committed ncu summary, if it was captured on this exact kernel source;
    null otherwise.  The key dominates and is read once per launch, so the
    figure does not scale with the bootstraps a launch processes."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        src = open(os.path.join(ROOT, "paper_2506_12761_gb300", "csrc", kernel_src), "rb").read()
        ent = rec.get(kernel_src)
        if ent and ent.get("sha256") == hashlib.sha256(src).hexdigest():
            return ent["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


_ORACLE = {}


def cpu_oracle_rate(budget_s: float = 20.0):
    """Oracle bootstraps/s on the host cores on a bounded sample of the same
    workload: the first-layer gates of the IntV circuit (the first ripple
    gate of each entry's four comparators), OpenMP over independent gates."""
    import oracle
    from paper_2506_12761_gb300 import synth
    if "keys" not in _ORACLE:
        _ORACLE["keys"] = oracle.keygen(oracle.paper_params(), synth.key_material())
    keys = _ORACLE["keys"]
    w = synth.intv_workload(D)
    lm_x = synth.lwe_material(32, seed=synth.MASTER_SEED, substream=1)
    lm_y = synth.lwe_material(32, seed=synth.MASTER_SEED, substream=2)
    cx = oracle.encrypt_bits(keys.s, synth.value_bits([w["x"]], 32)[0], lm_x)
    cy = oracle.encrypt_bits(keys.s, synth.value_bits([w["y"]], 32)[0], lm_y)
    threads = oracle.default_threads()
    n = 630
    t_le = oracle.trivial(n, 1 << 29)                # HomCompLE starts from Enc(1)
    t_lt = oracle.trivial(n, (1 << 32) - (1 << 29))  # HomCompL starts from Enc(0)
    groups = {}
    for d in range(D):
        r = [int(v) for v in w["rects"][d]]
        for ct, lo, hi in ((cx, r[0], r[1]), (cy, r[2], r[3])):
            groups.setdefault(oracle.AND if lo & 1 else oracle.OR, []).append(np.stack([ct[0], t_le]))
            groups.setdefault(oracle.ORNY if hi & 1 else oracle.ANDNY, []).append(np.stack([ct[0], t_lt]))
    order = [(g, x) for g, items in groups.items() for x in items]
    per_call = 2 * threads
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget_s and done < len(order):
        chunk = order[done:done + per_call]
        for g in {g for g, _ in chunk}:
            oracle.gate_batch(keys, g, np.stack([x for gg, x in chunk if gg == g]), threads=threads)
        done += len(chunk)
    dt = time.perf_counter() - t0
    return done / dt, threads, (f"{done} first-layer gate bootstraps of the D=1024 IntV workload "
                                f"(OpenMP over gates, {threads} threads) in {dt:.1f} s")


def cpu_oracle_config1():
    """The oracle's whole identifier-matching circuit of the small workload
    (8-bit id, D = 4 ids, 28 bootstraps in AND-tree layers of 16, 8 and 4),
    timed exactly on the host cores."""
    import oracle
    from paper_2506_12761_gb300 import synth
    if "keys" not in _ORACLE:
        _ORACLE["keys"] = oracle.keygen(oracle.paper_params(), synth.key_material())
    keys = _ORACLE["keys"]
    w = synth.idm_workload(4, 8)
    x = oracle.encrypt_bits(keys.s, synth.value_bits([w["query"]], 8)[0], synth.lwe_material(8, substream=31))
    t0 = time.perf_counter()
    out = oracle.idm_batch(keys, x, w["ids"].astype(np.uint64))
    dt = time.perf_counter() - t0
    ok = list(oracle.decrypt_bits(keys.s, out)) == [int(i == w["query"]) for i in w["ids"]]
    return {"bootstraps": 28, "seconds": dt, "value": 28 / dt, "unit": UNIT, "decrypt_ok": ok,
            "threads": oracle.default_threads(),
            "workload": "identifier matching, 8-bit encrypted id vs D=4 plaintext ids (28 bootstraps), whole circuit"}


def bench_config(world: int) -> dict:
    """The `config` record, identical in both arms (what each arm timed of the
    workload is stated beside it, under "run")."""
    return {"workload": WORKLOAD, "D": D, "bootstraps_per_step": BOOTSTRAPS_PER_STEP,
            "parallelism": f"replicas x{world}",
            "l2": "GPU arm: L2 flushed between timed steps (256 MiB write, untimed); the CPU arm has no GPU cache"}


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    steps = []
    info = None
    for _ in range(args.warmup + args.steps):
        r, cores, sample = cpu_oracle_rate(budget_s=args.ref_budget)
        steps.append(r)
        info = (cores, sample)
    vals = steps[args.warmup:]
    v = float(np.mean(vals))
    sample = ("each step: a bounded sample of the workload, " + info[1] +
              "; ms_per_step extrapolated to the whole query as bootstraps_per_step / rate")
    c1 = cpu_oracle_config1()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": BOOTSTRAPS_PER_STEP / v * 1e3,
            "ms_per_step_basis": "extrapolated from the timed sample (a full CPU query takes about an hour)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": bench_config(world), "run": {"sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": info[0], "kind": "oracle", "sample": info[1],
                             "config1_full_circuit": c1},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_wave(args):
    """One-launch measurement of the blind-rotation kernel: `--wave` AND gates
    in one velopir_bootstrap_batch call, `--warmup` untimed then `--steps`
    timed, with the library's CUDA-event profiler around each launch.  A count
    of 152 x W is one full wave of the W-wide tile shape (1,824 fills every SM
    with 12 bootstraps).  This is the command the kernel profiles capture."""
    import torch
    from paper_2506_12761_gb300 import build, synth
    from paper_2506_12761_gb300 import velopir as vp
    build.build()
    km = synth.key_material()
    bk, ksk = vp.velopir_client_keygen(km)
    ctx = vp.Context(0)
    vp.velopir_load_cloud_key(ctx.h, bk, ksk)
    vp.velopir_set_path(ctx.h, {"dense": vp.VP_PATH_INT32_DENSE, "ntt": vp.VP_PATH_NTT,
                                 "tensor": vp.VP_PATH_TENSOR_F16}[args.path])
    n = args.wave
    bits = synth.Stream(synth.MASTER_SEED, synth.STREAM_QUERY, 9).bits(n * 2)
    ct = vp.velopir_client_encrypt_bits(km.s, bits, synth.lwe_material(n * 2, substream=9)).reshape(n, 2, 631)
    din = torch.from_numpy(ct.view(np.int32)).cuda()
    dout = torch.zeros((n, 631), dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        vp.velopir_bootstrap_batch(ctx.h, vp.VP_AND, din, dout, n)
    vp.velopir_profile(ctx.h, True)
    per = []
    for _ in range(args.steps):
        b0 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_BLIND_ROTATE)
        k0 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_KEY_SWITCH)
        vp.velopir_bootstrap_batch(ctx.h, vp.VP_AND, din, dout, n)
        b1 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_BLIND_ROTATE)
        k1 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_KEY_SWITCH)
        per.append({"br_launches": b1[0] - b0[0], "br_ms": b1[2] - b0[2], "ks_ms": k1[2] - k0[2]})
    vp.velopir_profile(ctx.h, False)
    b = bits.reshape(-1, 2)
    ok = bool(np.array_equal(vp.velopir_client_decrypt_bits(km.s, dout.cpu().numpy().view(np.uint32)),
                             b[:, 0] & b[:, 1]))
    best = min(p["br_ms"] for p in per)
    print(json.dumps({"mode": "one launch", "path": args.path, "count": n, "launches": per,
                      "blind_rotations_per_s": n / (best / 1e3), "decrypt_ok": ok}), flush=True)
    ctx.close()
    return 0 if ok else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="ntt", choices=["dense", "ntt", "tensor"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--latency-queries", type=int, default=20)
    ap.add_argument("--wave", type=int, default=0,
                    help="instead of the query: one batch of this many AND gates per step (kernel profiles)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.wave:
        return run_wave(args)

    import torch
    from paper_2506_12761_gb300 import build, synth
    from paper_2506_12761_gb300 import velopir as vp

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    dist = Dist(world)
    build.build()

    # keys and query from the library's own client code (no oracle on this path)
    km = synth.key_material()
    bk, ksk = vp.velopir_client_keygen(km)
    stream = torch.cuda.current_stream()
    ctx = vp.Context(local, 0, stream.cuda_stream)
    vp.velopir_load_cloud_key(ctx.h, bk, ksk)
    vp.velopir_set_path(ctx.h, {"dense": vp.VP_PATH_INT32_DENSE, "ntt": vp.VP_PATH_NTT,
                                 "tensor": vp.VP_PATH_TENSOR_F16}[args.path])
    waves = vp.velopir_autotune(ctx.h) if args.path == "ntt" else []   # tile-shape autotuner (untimed set-up)
    w = synth.intv_workload(D, substream=rank)
    cx = vp.velopir_client_encrypt_bits(km.s, synth.value_bits([w["x"]], 32)[0], synth.lwe_material(32, substream=1 + 2 * rank))
    cy = vp.velopir_client_encrypt_bits(km.s, synth.value_bits([w["y"]], 32)[0], synth.lwe_material(32, substream=2 + 2 * rank))
    rects = np.ascontiguousarray(w["rects"], dtype=np.uint32)
    dx = torch.from_numpy(cx.view(np.int32)).cuda()
    dy = torch.from_numpy(cy.view(np.int32)).cuda()
    dr = torch.from_numpy(rects.view(np.int32)).cuda()
    dout = torch.zeros((D, 631), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    def step():
        vp.velopir_interval_query(ctx.h, dx, dy, dr, D, dout)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of the last warm-up output against the plaintext predicate
    got = vp.velopir_client_decrypt_bits(km.s, dout.cpu().numpy().view(np.uint32))
    r64 = rects.astype(np.int64)
    want = ((r64[:, 0] <= w["x"]) & (w["x"] < r64[:, 1]) & (r64[:, 2] <= w["y"]) & (w["y"] < r64[:, 3])).astype(np.uint32)
    decrypt_ok = bool(np.array_equal(got, want))

    clocks = Clocks(local)
    vp.velopir_profile(ctx.h, True)
    launches0 = vp.velopir_launch_count(ctx.h)
    dist.barrier()
    torch.cuda.synchronize()
    per_step = []
    for _ in range(args.steps):
        flush.random_()   # evict L2 between timed steps (untimed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        per_step.append(e0.elapsed_time(e1))
    dist.barrier()
    launches = vp.velopir_launch_count(ctx.h) - launches0
    n_br, u_br, ms_br = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_BLIND_ROTATE)
    n_ks, u_ks, ms_ks = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_KEY_SWITCH)
    vp.velopir_profile(ctx.h, False)
    clk = clocks.stop()
    t_total = dist.max(sum(per_step) / 1e3)
    value = world * args.steps * BOOTSTRAPS_PER_STEP / t_total

    # end to end through the public API with pinned host buffers (H2D + D2H inside the timed region)
    hx = torch.from_numpy(cx.view(np.int32)).pin_memory()
    hy = torch.from_numpy(cy.view(np.int32)).pin_memory()
    hr = torch.from_numpy(rects.view(np.int32)).pin_memory()
    hout = torch.zeros((D, 631), dtype=torch.int32).pin_memory()
    e2e_t = []
    dist.barrier()
    for _ in range(max(1, args.steps)):
        flush.random_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vp.velopir_interval_query(ctx.h, hx, hy, hr, D, hout)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = dist.max(sum(e2e_t))
    e2e_value = world * len(e2e_t) * BOOTSTRAPS_PER_STEP / e2e_total
    h2d = (cx.nbytes + cy.nbytes + rects.nbytes)
    d2h = D * 631 * 4

    # plain: one bootstrap per kernel launch, same kernels (one warm-up pass, then repeats)
    plain_n = 8 if args.path == "dense" else 64
    bits = synth.Stream(5, 2, 99).bits(2 * plain_n)
    pin = vp.velopir_client_encrypt_bits(km.s, bits, synth.lwe_material(2 * plain_n, seed=5)).reshape(plain_n, 2, 631)
    dpin = torch.from_numpy(pin.view(np.int32)).cuda()
    dpout = torch.zeros((plain_n, 631), dtype=torch.int32, device="cuda")
    vp.velopir_bootstrap_plain(ctx.h, vp.VP_AND, dpin[:4], dpout[:4], 4)
    plain_rates = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vp.velopir_bootstrap_plain(ctx.h, vp.VP_AND, dpin, dpout, plain_n)
        torch.cuda.synchronize()
        plain_rates.append(plain_n / (time.perf_counter() - t0))
    plain_rate = float(np.median(plain_rates))

    # query latency of the small identifier-matching workload (8-bit id, D = 4,
    # 28 bootstraps): layer-batched launches against one bootstrap per launch
    w1 = synth.idm_workload(4, 8)
    x1 = torch.from_numpy(vp.velopir_client_encrypt_bits(km.s, synth.value_bits([w1["query"]], 8)[0],
                                                         synth.lwe_material(8, substream=31)).view(np.int32)).cuda()
    ids1 = torch.from_numpy(w1["ids"].astype(np.uint32).view(np.int32)).cuda()
    out1 = torch.zeros((4, 631), dtype=torch.int32, device="cuda")
    lat = {}
    for mode, limit in (("batched", 0), ("plain", 1)):
        vp.velopir_set_launch_limit(ctx.h, limit)
        vp.velopir_id_match(ctx.h, x1, 8, ids1, 4, None, 0, out1)     # warm-up
        ts = []
        for _ in range(args.latency_queries):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            vp.velopir_id_match(ctx.h, x1, 8, ids1, 4, None, 0, out1)
            ts.append((time.perf_counter() - t0) * 1e3)
        ok = list(vp.velopir_client_decrypt_bits(km.s, out1.cpu().numpy().view(np.uint32))) == \
            [int(i == w1["query"]) for i in w1["ids"]]
        lat[mode] = {"p50": float(np.percentile(ts, 50)), "p99": float(np.percentile(ts, 99)), "queries": len(ts),
                     "decrypt_ok": ok}
    vp.velopir_set_launch_limit(ctx.h, 0)

    # roofline of the dominant kernel (blind rotation), timed live above
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    if args.path == "tensor":
        kernel_src = "br_tc.cu"
        # fp16 MMA work: 4 key limbs x the dense contraction, 2 flops per multiply-add
        achieved = (u_br * 4 * MACS_DENSE * 2) / (ms_br / 1e3) / 1e12
        peak = peaks.get("bf16_tflops", 1900.0)   # fp16 and bf16 dense rates are equal
        unit = "TFLOP/s"
    elif args.path == "dense":
        kernel_src = "br_dense.cu"
        achieved = (u_br * MACS_DENSE) / (ms_br / 1e3) / 1e12
        peak = 152 * 64 * sm_max * 1e6 / 1e12   # int32 multiply-add pipe: 64 lanes/clk/SM
        unit = "T int32-MAC/s"
    else:
        kernel_src = "br_ntt.cu"
        from paper_2506_12761_gb300 import ntt_model
        # a high-half multiply holds the 64-lane IMAD pipe for two slots (measured; see ntt_model)
        achieved = (u_br * ntt_model.IMAD_SLOTS_PER_BOOTSTRAP) / (ms_br / 1e3) / 1e12
        peak = 152 * 64 * sm_max * 1e6 / 1e12
        unit = "T IMAD lane-slots/s"
    roofline = {"bound": "tensor" if args.path == "tensor" else "alu", "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak,
                "traffic": traffic_for(kernel_src),
                "kernel": kernel_src.replace(".cu", ""), "launches": n_br, "avg_launch_ms": ms_br / max(1, n_br),
                "peak_basis": ("measured cuBLAS bf16 dense GEMM (MEASURED_PEAKS.json bf16_tflops)"
                               if args.path == "tensor" else
                               "152 SMs x 64 int32 multiply lanes/clk x max SM clock %.0f MHz" % sm_max),
                "work_per_bootstrap": ({"imad_slots": ntt_model.IMAD_SLOTS_PER_BOOTSTRAP,
                                        "multiplies": ntt_model.IMAD_OPS_PER_BOOTSTRAP,
                                        "slot_rule": "low-half multiply 1 slot, high-half multiply 2 slots"}
                                       if args.path == "ntt" else {"int32_macs": MACS_DENSE}),
                "key_switch": {"launches": n_ks, "avg_launch_ms": ms_ks / max(1, n_ks),
                               "share_of_step": ms_ks / max(1e-9, sum(per_step))}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, sample = cpu_oracle_rate()
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "config1_full_circuit": cpu_oracle_config1()}

    if rank == 0:
        ms = [float(x) for x in per_step]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": bench_config(world),
                "run": {"sample": "each step: the whole query, every bootstrap of it", "path": args.path,
                        "tile_shapes": {"wave_ms_by_bootstraps_per_cta": dict(zip(vp.NTT_TILE_SHAPES, waves))}},
                "query_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
                "plain": {"value": plain_rate, "unit": UNIT, "repeats": [float(x) for x in plain_rates],
                          "note": "one bootstrap per kernel launch, same kernels; median of 3 passes after a warm-up"},
                "config1_query_ms": dict(lat, workload="identifier matching, 8-bit id vs D=4 ids, 28 bootstraps",
                                         note="batched: gate layers as launches; plain: one bootstrap per launch"),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
                "decrypt_ok": decrypt_ok}
        print(json.dumps(line), flush=True)
    ctx.close()
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
