"""Compile the C oracle (``sv_oracle.c``) into ``liboracle.so`` next to it.

Test infrastructure: called by ``__graft_entry__.build()`` and, on demand, by
``oracle.oracle`` when the shared object is missing or older than its source.
Plain ISO C11 with no fast-math and no FMA contraction, so the oracle rounds
as the C source reads; OpenMP parallelises the gate loop when the compiler
has it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sv_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", SRC]
    tmp = LIB + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = base + extra + ["-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
        if verbose:
            print(r.stderr, file=sys.stderr)
    raise RuntimeError("could not compile the oracle: " + r.stderr)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
