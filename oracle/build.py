"""Compile the oracle's C core (fci.c) into a host shared library with gcc.

Test infrastructure only: the CUDA product path never loads this library.
Plain portable C (no x86 or Arm intrinsics), so the same source builds on the
x86 development container and on the Arm GPU host.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fci.c")
LIB = os.path.join(HERE, "_oracle_fci.so")


def build(force: bool = False) -> str:
    """Build oracle/_oracle_fci.so if it is missing or older than fci.c."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
