"""Relative throughput of the integer multiply streams (csrc/int_peak.cu):
32-bit low multiply-adds, high multiplies and Shoup modular products, each
as independent chains filling every SM, timed with the SM's clock64 counter
back to back.  The blind-rotation roofline counts a low multiply as one
lane-slot and a high multiply as two, so a Shoup product (one high, two low)
as four; the ratios printed here are what that rule asserts, measured.

    python -m paper_2506_12761_gb300.int_peak
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

from . import build

HERE = os.path.dirname(os.path.abspath(__file__))


def main() -> int:
    exe = os.path.join(build.BUILD, "int_peak")
    os.makedirs(build.BUILD, exist_ok=True)
    src = os.path.join(HERE, "csrc", "int_peak.cu")
    r = subprocess.run([build.nvcc(), "-std=c++17", "-O3", *build.ARCH, src, "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        return 1
    r = subprocess.run([exe], capture_output=True, text=True)
    rates = {}
    for line in r.stdout.splitlines():
        d = json.loads(line)
        if "op" in d:
            rates[d["op"]] = d["lane_ops_per_tick_per_sm"]
        print(line, flush=True)
    if r.returncode != 0 or len(rates) != 3:
        return 1
    print(json.dumps({"low_multiplies_per_high_multiply": rates["lo"] / rates["hi"],
                      "low_multiplies_per_shoup_product": rates["lo"] / rates["shoup"]}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
