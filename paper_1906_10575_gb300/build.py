"""Builds libamgdd.so in-tree: CUDA kernels for sm_103a plus the host setup.

nvcc compiles the kernels (-fmad=false: only explicit fma() calls fuse, which
keeps every row product the fixed ascending fma chain); g++ compiles the host
setup with -ffp-contract=off so the hierarchy is identical on x86 and Arm.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libamgdd.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")

CU_SOURCES = ["kernels.cu", "kernels_multi.cu", "fac_multi_r1.cu", "fac_multi_r2.cu", "fac_multi_r4.cu",
              "fac_vsm.cu", "fac_cluster.cu", "adjoint.cu", "noalloc.cu"]
CXX_SOURCES = ["hierarchy.cpp", "composite.cpp", "capi.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh"))
    ] + [os.path.join(os.path.dirname(HERE), "include", "amgdd.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + os.path.join(CUDA_HOME, "include"), "-I" + CSRC]
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([NVCC, ARCH, "-O3", "-std=c++17", "-fmad=false", "-lineinfo", "-Xptxas", "-v",
                     "-Xcompiler", "-fPIC", "-c", os.path.join(CSRC, f), "-o", o] + inc)
    for f in CXX_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
                     "-Wall", "-Wno-unused-function", "-c", os.path.join(CSRC, f), "-o", o] + inc)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".%d.tmp" % os.getpid()
    _run([NVCC, ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs + ["-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
