"""Measure the GB300 arithmetic throughputs the rooflines refer to.

python -m paper_1012_5082_gb300.alu_peaks  -> one JSON line (per GPU):
FP64/FP32 FMA, FP64 exp, FP32 expf, tanh.approx, INT32 xor+add, popc,
32-bit mul.hi + mul.lo pairs and legacy mma.sync BF16 throughput.
"""
import subprocess
import sys

from . import build


def main() -> int:
    exe = build.build_alu_peaks()
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    sys.stderr.write(r.stderr)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
