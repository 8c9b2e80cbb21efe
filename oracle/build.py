"""Compile the CPU oracle into oracle/liboracle.so (g++, OpenMP).

Test infrastructure: the oracle checks the CUDA library; the library never
loads it.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["ckks_oracle.cpp", "oracle_layers.cpp"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle_internal.h", os.path.join("..", "inputs", "he_random.h")]
    return any(os.path.getmtime(os.path.join(HERE, d)) > t for d in deps)


def build(force: bool = False) -> str:
    if force or _stale():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + \
              [os.path.join(HERE, s) for s in SOURCES]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
