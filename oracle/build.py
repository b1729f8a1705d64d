"""Build the C oracle (3D and 2D) into oracle/_build/libma_oracle.so with gcc.

Test infrastructure: the oracle is the checker the CUDA library is compared
with.  Building it is not using it; only tests, the smoke check and the
benchmark's CPU-baseline leg load the result.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
SRC = HERE / "ma_oracle.c"
SRCS = [SRC, HERE / "ma2d_oracle.c"]
OUT_DIR = HERE / "_build"
LIB = OUT_DIR / "libma_oracle.so"


def build(force: bool = False) -> Path:
    """Compile the oracle (FP64, -O2, OpenMP within a colour) if it is stale."""
    OUT_DIR.mkdir(exist_ok=True)
    if not force and LIB.exists() and all(LIB.stat().st_mtime >= s.stat().st_mtime for s in SRCS):
        return LIB
    tmp = OUT_DIR / f"libma_oracle.{os.getpid()}.so"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
           "-o", str(tmp), *[str(s) for s in SRCS], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
