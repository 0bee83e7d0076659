"""Compile the FP64 CPU oracle (psolve_oracle.c) into shared libraries beside it.

Flags: -O2 with IEEE semantics (-ffp-contract=off, no -ffast-math) so that
the error-free transformations of the compensated dot product hold.

Two builds of the same source:
  liboracle.so      serial (no OpenMP, no SIMD intrinsics): the parity oracle;
  liboracle_omp.so  -fopenmp, loops spread with a static schedule and the dot
                    product summed over fixed index ranges (independent of the
                    thread count): the timed CPU baseline and long stored runs.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "psolve_oracle.c")
LIB_PATH = os.path.join(HERE, "liboracle.so")
LIB_OMP_PATH = os.path.join(HERE, "liboracle_omp.so")


def _compile(out: str, extra: list[str], force: bool) -> str:
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "psolve_oracle.h")),
            os.path.getmtime(os.path.abspath(__file__))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", *extra, "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """The serial oracle (the parity reference)."""
    return _compile(LIB_PATH, [], force)


def build_omp(force: bool = False) -> str:
    """The OpenMP build of the same source."""
    return _compile(LIB_OMP_PATH, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_omp(force=True))
