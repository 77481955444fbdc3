"""Compile the oracle's C part (``netsimplex.c``) into ``oracle/_build/liboracle.so``.

Test infrastructure only (see ``oracle/__init__.py``).  Plain gcc, no architecture flags,
so the same source builds on x86-64 and aarch64.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SOURCES = [os.path.join(HERE, "netsimplex.c")]


def build(force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(LIB) for s in SOURCES)
    if stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, *SOURCES, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
