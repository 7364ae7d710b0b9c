"""Build and run the tensor-core issue-rate probe (csrc/mma_rate.cu, a stand-alone
program): cycles per tcgen05.mma for several tile shapes, with a runtime-bounded and a
fully unrolled issue loop, and cycles per warp-level mma.sync m16n8k16.  These rates set
the tile and instruction choices of the H-apply and the block-update kernels.

Usage: python -m paper_2111_02534_gb300.mma_rate
"""
from __future__ import annotations

import os
import subprocess
import sys

from .build import ARCH, BUILD_DIR, CSRC, _nvcc


def main() -> int:
    os.makedirs(BUILD_DIR, exist_ok=True)
    exe = os.path.join(BUILD_DIR, "mma_rate")
    cmd = [_nvcc(), "-std=c++17", "-O3"] + ARCH + ["-I", CSRC, os.path.join(CSRC, "mma_rate.cu"),
                                                  "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        return r.returncode
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
