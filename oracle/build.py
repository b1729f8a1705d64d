"""Build the C oracle into oracle/_build/libma_oracle.so with gcc.

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
OUT_DIR = HERE / "_build"
LIB = OUT_DIR / "libma_oracle.so"


def build(force: bool = False) -> Path:
    """Compile the oracle (FP64, -O2, OpenMP within a colour) if it is stale."""
    OUT_DIR.mkdir(exist_ok=True)
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = OUT_DIR / f"libma_oracle.{os.getpid()}.so"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
           "-o", str(tmp), str(SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
