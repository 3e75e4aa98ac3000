"""Compile the CPU oracle (plain C) into oracle/_build/liboracle.so.

Test infrastructure: called by the tests, the smoke check, the benchmark's
CPU-baseline leg and the package build step (building the checker is not
using it).  Plain gcc; OpenMP is used when the compiler accepts it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", SRC, "-lm"]
    tmp = LIB + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:] + ["-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
        if verbose:
            print(r.stderr, file=sys.stderr)
    raise RuntimeError("failed to build the CPU oracle: " + r.stderr)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
