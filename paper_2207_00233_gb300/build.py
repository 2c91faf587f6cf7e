"""Build ``libfse_gb300.so`` in-tree for sm_103a.

The CUDA translation unit is compiled by nvcc for ``sm_103a`` only; the host
runtime by g++.  Objects compile in parallel; nothing uses cmake.
Run ``python -m paper_2207_00233_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfse_gb300.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["fse_kernels.cu", "fse_noalloc.cu", "fse_peaks.cu", "fse_loopbench.cu",
              "fse_wtable_tc.cu"]
CPP_SOURCES = ["fse_api.cpp", "fse_hostbatch.cpp", "fse_serve.cpp", "fse_plan.cpp", "fse_sched.cpp"]
HEADERS = ["fse_internal.h", "fse_ctx.h", "fse_iter.cuh"]


def _inputs():
    paths = [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES + HEADERS]
    paths.append(os.path.join(INCLUDE, "fse.h"))
    paths.append(os.path.abspath(__file__))
    return paths


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of the shared library."""
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cxx = shutil.which("g++") or "g++"
    jobs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, src))
        objs.append(obj)
    for src in CPP_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
               "-I", INCLUDE, "-I", os.path.join(CUDA_HOME, "include"), "-c",
               os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, src))
        objs.append(obj)
    procs = [(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src)
             for cmd, src in jobs]
    failed = []
    for p, src in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip():
            print(f"--- {src}\n{text}")
    if failed:
        msg = "\n".join(f"--- {s}\n{t}" for s, t in failed)
        raise RuntimeError(f"build of libfse_gb300.so failed:\n{msg}")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [NVCC, "-shared", *ARCH, "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    subprocess.run(link, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
