"""Compile the C part of the oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain gcc, no machine-specific flags, and no floating-point contraction so that
the oracle gives the same bits on x86_64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sme_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
# The same source built with OpenMP: the timed CPU baseline on all host cores (same bits, see sme_oracle.c).
LIB_OMP = os.path.join(OUT_DIR, "liboracle_omp.so")


def _build(out: str, flags, force: bool) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *flags, "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_oracle(force: bool = False) -> str:
    """The checker: single-threaded -O2."""
    return _build(LIB, ["-O2"], force)


def build_oracle_omp(force: bool = False) -> str:
    """The timed baseline: -O3 with OpenMP over rows, columns and probe-table entries."""
    return _build(LIB_OMP, ["-O3", "-fopenmp"], force)


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
    print(build_oracle_omp(force="--force" in sys.argv))
