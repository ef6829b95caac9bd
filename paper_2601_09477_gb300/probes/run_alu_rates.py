"""Build and run alu_rates.cu on the current GPU and print its JSON line.

The rates it measures (FP32, packed FP32x2 and FP64 adds, 32/64-bit integer
adds, integer multiply-add, conversions, shared-memory integer atomics) are
the per-SM issue rates the sketch kernels' rooflines are stated against.

Usage: python -m paper_2601_09477_gb300.probes.run_alu_rates [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(os.path.dirname(HERE), "_build")


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="also write the JSON line to this file")
    a = ap.parse_args()
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "alu_rates")
    src = os.path.join(HERE, "alu_rates.cu")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    if out.returncode != 0:
        sys.stderr.write(out.stderr)
        return out.returncode
    line = out.stdout.strip().splitlines()[-1]
    json.loads(line)   # well-formed
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
