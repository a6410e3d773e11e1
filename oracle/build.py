"""Compile the FP64 CPU oracle into oracle/liboracle.so (plain gcc, no CUDA).

Test infrastructure only: the oracle is built so that tests, the smoke check
and the CPU-baseline leg of the benchmark can load it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["forcefield.c", "minimizers.c", "mlp.c"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    hdr = os.path.join(HERE, "ffmin_oracle.h")
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr, __file__])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra", "-Wdouble-promotion", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
