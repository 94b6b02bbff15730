"""One-launch measurement of the blind-rotation kernel: `count` AND gates in a
single velopir_bootstrap_batch call, repeated `--reps` times.

A count of 152 x W on the NTT path is one full wave of the W-wide tile shape
(1,824 = 152 x 12 fills every SM with 12 bootstraps).  Per launch it prints
the blind-rotation and key-switch device times from the library's own
CUDA-event profiler and checks every output bit against the plaintext AND.
This is the driver of the per-kernel profiles:

    python -m paper_2506_12761_gb300.wave_bench --path ntt --count 1824 --tune
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import build, synth
from . import velopir as vp


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--path", choices=("ntt", "dense"), default="ntt")
    ap.add_argument("--count", type=int, default=1824)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tune", action="store_true", help="run the tile-shape autotuner first (NTT path)")
    args = ap.parse_args()

    import torch
    build.build()
    km = synth.key_material()
    bk, ksk = vp.velopir_client_keygen(km)
    ctx = vp.Context(0)
    vp.velopir_load_cloud_key(ctx.h, bk, ksk)
    vp.velopir_set_path(ctx.h, {"dense": vp.VP_PATH_INT32_DENSE, "ntt": vp.VP_PATH_NTT}[args.path])
    waves = vp.velopir_autotune(ctx.h) if args.tune and args.path == "ntt" else None

    n = args.count
    bits = synth.Stream(synth.MASTER_SEED, synth.STREAM_QUERY, 9).bits(n * 2)
    ct = vp.velopir_client_encrypt_bits(km.s, bits, synth.lwe_material(n * 2, substream=9)).reshape(n, 2, 631)
    din = torch.from_numpy(ct.view(np.int32)).cuda()
    dout = torch.zeros((n, 631), dtype=torch.int32, device="cuda")
    vp.velopir_profile(ctx.h, True)
    per = []
    for _ in range(args.reps):
        b0 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_BLIND_ROTATE)
        k0 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_KEY_SWITCH)
        vp.velopir_bootstrap_batch(ctx.h, vp.VP_AND, din, dout, n)
        b1 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_BLIND_ROTATE)
        k1 = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_KEY_SWITCH)
        per.append({"br_launches": b1[0] - b0[0], "br_ms": b1[2] - b0[2], "ks_ms": k1[2] - k0[2]})
    b = bits.reshape(-1, 2)
    ok = bool(np.array_equal(vp.velopir_client_decrypt_bits(km.s, dout.cpu().numpy().view(np.uint32)),
                             b[:, 0] & b[:, 1]))
    best = min(p["br_ms"] for p in per)
    print(json.dumps({"path": args.path, "count": n, "tile_shape": vp.velopir_tuned_shape(ctx.h, n) if waves else None,
                      "autotune_wave_ms": waves, "launches": per,
                      "blind_rotations_per_s": n / (best / 1e3), "decrypt_ok": ok}))
    ctx.close()
    if not ok:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
