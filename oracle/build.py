"""Compile the C oracle into oracle/liboracle.so (test infrastructure)."""
from __future__ import annotations

import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["sph_oracle.c", "sph_oracle_adjoint.c", "sph_oracle_bc.c", "sph_oracle_dem.c"]
LIB = os.path.join(_HERE, "liboracle.so")

# ISO C mode keeps floating-point contraction off; -ffp-contract=off makes it
# explicit.  No -march flags: the same source builds on x86-64 and aarch64.
CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
          "-shared", "-D_DEFAULT_SOURCE"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for s in SOURCES + ["build.py", "sph_oracle_bc.h"]:
        p = os.path.join(_HERE, s)
        if os.path.exists(p) and os.path.getmtime(p) > t:
            return True
    return False


def build(force: bool = False) -> str:
    if force or _stale():
        srcs = [os.path.join(_HERE, s) for s in SOURCES if os.path.exists(os.path.join(_HERE, s))]
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, "-o", tmp, *srcs, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stderr)
            raise RuntimeError("oracle build failed: " + " ".join(cmd))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
