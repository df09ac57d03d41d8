"""Compile the CPU oracle (plain C, OpenMP) into ``oracle/_lib/liboracle.so``.

Test infrastructure: building the checker is not using it.  Plain gcc, no
architecture-specific flags, so the same source builds on x86-64 and on Arm.
"""

from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.path.join(_HERE, "_lib", "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    out = lib_path()
    src = os.path.join(_HERE, "fmap_oracle.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
           "-fno-fast-math", "-ffp-contract=off", src, "-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
