"""Build and run umma_hadamard.cu on the current GPU and print its JSON line.

It times the 2^14-point Walsh-Hadamard transform of one slice as two
128 x 128 x 128 tensor-core products (tcgen05.mma, BF16 operands, FP32
accumulation), with and without the 16-bit rounding of the intermediate and
the shared-memory pass a sketch kernel would add, and checks one slice against
the exact transform.

Usage: python -m paper_2601_09477_gb300.probes.run_umma_hadamard [--out FILE]
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
    ap.add_argument("--iters", type=int, default=2000, help="slices per CTA in the timed launch")
    a = ap.parse_args()
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "umma_hadamard")
    src = os.path.join(HERE, "umma_hadamard.cu")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-o", exe, src], check=True)
    out = subprocess.run([exe, str(a.iters)], capture_output=True, text=True, timeout=300)
    if out.returncode != 0:
        sys.stderr.write(out.stdout + out.stderr)
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
