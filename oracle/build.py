"""Compile the C oracle into ``oracle/liboracle.so`` (test infrastructure).

Plain gcc, FP64, ``-O2 -ffp-contract=off`` (no fused multiply-adds, every
expression evaluated as written), OpenMP across systems only.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ode_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_LIBM = os.path.join(HERE, "liboracle_libm.so")


def build(force: bool = False, libm: bool = False) -> str:
    """The oracle library; libm=True builds the comparison variant whose
    powers come from the C library instead of the series of reading R10."""
    lib = LIB_LIBM if libm else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", *(["-DORACLE_LIBM"] if libm else []), "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, libm="--libm" in sys.argv))
