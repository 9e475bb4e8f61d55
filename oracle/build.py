"""Compile the plain-C oracle into ``oracle/_build/libspin_oracle.so`` with gcc.

Test infrastructure: the product never runs this.  ``-ffp-contract=off`` keeps
gcc from fusing multiply-adds, so x86-64 and aarch64 builds round alike.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
SRC = HERE / "spin_oracle.c"
OUT_DIR = HERE / "_build"
LIB = OUT_DIR / "libspin_oracle.so"


def build(force: bool = False, verbose: bool = False) -> Path:
    """Build the oracle shared library if it is missing or older than its source."""
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    OUT_DIR.mkdir(parents=True, exist_ok=True)
    tmp = OUT_DIR / f"libspin_oracle.{os.getpid()}.so"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", str(tmp), str(SRC), "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
