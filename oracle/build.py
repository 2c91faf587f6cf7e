"""Compile the FP64 CPU oracle into ``oracle/liboracle_fse.so`` with gcc.

Test infrastructure only.  Built with ``-ffp-contract=off`` so that no
fused multiply-add changes its rounding between x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fse_oracle.c")
HDR = os.path.join(HERE, "fse_oracle.h")
LIB = os.path.join(HERE, "liboracle_fse.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    mtime = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > mtime for p in (SRC, HDR, __file__))


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra",
               "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
