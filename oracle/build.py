"""Compile the FP64 oracle (plain C) into oracle/liboracle.so.

Test infrastructure: the oracle is built by the same build step as the CUDA
library, but only tests, the smoke check and the benchmark's CPU-baseline leg
load it.  -ffp-contract=off keeps every operation a separate IEEE rounding on
both x86-64 and aarch64 (gcc contracts to FMA by default on aarch64).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
