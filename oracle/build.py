"""Compile the CPU oracle (plain C, gcc, OpenMP) into oracle/_build/.

Test infrastructure: the oracle is built so the tests, the smoke check and
the bench's CPU-baseline leg can call it; the product path never links it.
Run as ``python oracle/build.py`` or through ``__graft_entry__.build()``.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hdc_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libhdc_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    # -ffp-contract=off keeps the double-double error-free transforms exact
    # on compilers that would otherwise fuse a*b+c (aarch64 gcc does).
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fvisibility=hidden", SRC, "-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
