"""Measure the FP32-FMA, FP64-FMA and MUFU-rsqrt peaks of the local GPU.

Compiles csrc/alu_peaks.cu for sm_103a and prints one JSON line.  These are
the denominators of the ALU rooflines reported by bench.py.
Usage: python -m paper_1905_04065_gb300.alu_peaks
"""
import os
import subprocess
import sys

from .build import ARCH, BUILD, CSRC, nvcc


def main() -> int:
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "alu_peaks")
    src = os.path.join(CSRC, "alu_peaks.cu")
    subprocess.run([nvcc()] + ARCH + ["-O3", "-o", exe, src], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
