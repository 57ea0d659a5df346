"""Build and run the radix-16 measurement: 16-point DFTs on the CUDA cores
(the FFT engine's butterfly) and on the tensor cores (FP16 and BF16 hi/lo splits,
mma.sync), with their errors against an FP64 DFT.

    python -m paper_2510_10070_gb300.a10.run [--blocks 1216] [--reps 64]

Prints one JSON line.  Needs nvcc and a GB300 (sm_103a).
"""

from __future__ import annotations

import argparse
import json
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dft16_mma.cu")
OUT = os.path.join(HERE, "_build", "dft16_mma")


def build() -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < os.path.getmtime(SRC):
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "--expt-relaxed-constexpr", "-o", OUT, SRC], check=True)
    return OUT


def run(blocks: int = 152 * 8, reps: int = 64) -> dict:
    exe = build()
    out = subprocess.run([exe, str(blocks), str(reps)], check=True, capture_output=True, text=True).stdout
    return json.loads(out.strip().splitlines()[-1])


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--blocks", type=int, default=152 * 8)
    ap.add_argument("--reps", type=int, default=64)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.blocks, a.reps)))


if __name__ == "__main__":
    main()
