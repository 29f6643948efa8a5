"""Compile the C oracle into ``oracle/_build/libvqe_oracle.so`` with gcc.

TEST INFRASTRUCTURE: the oracle is built so the test suite, the smoke check
and the benchmark's CPU baseline can load it; the CUDA library never does.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vqe_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libvqe_oracle.so")


def _needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    newest = max(os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "vqe_oracle.h")))
    return os.path.getmtime(LIB) < newest


def build(force: bool = False) -> str:
    """Build the shared library if it is missing or stale; return its path."""
    if not force and not _needs_build():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)       # no OpenMP on this host: single thread
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
