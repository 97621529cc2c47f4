"""Compile the plain-C FP64 oracle into ``oracle/_build/libnb_oracle.so``.

Test infrastructure: the oracle is the checker of the CUDA path, never part of
it.  ``-ffp-contract=off`` keeps every multiply and add separately rounded so
the oracle's arithmetic is the plain order written in ``nb_oracle.c`` on both
x86-64 and AArch64 hosts.  It is built with OpenMP where the compiler has it:
the parallel loops are over independent elements, nodes or fixed chunks, so
the results do not depend on the number of threads.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nb_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libnb_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    # OpenMP spreads the element loop and the parallel PCG over the host
    # cores; a compiler without it builds the same code single-threaded.
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
