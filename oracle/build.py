"""Compile the FP64 CPU oracle into ``oracle/_build/liboracle.so`` (test infrastructure only).

gcc -O2 -fopenmp -ffp-contract=off: no fused multiply-adds, so the squared
distances that decide neighbour membership are plain IEEE products and sums.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SOURCES = ["af_oracle.c", "afmp_oracle.c", "gf_oracle.c"]
HEADERS = ["oracle_common.h"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t
               for f in SOURCES + HEADERS + [os.path.basename(__file__)]
               if os.path.exists(os.path.join(HERE, f)))


def build(force: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = [os.path.join(HERE, f) for f in SOURCES if os.path.exists(os.path.join(HERE, f))]
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
