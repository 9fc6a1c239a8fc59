"""Builds libmacroaim.so in-tree (sm_103a only), compiling translation units in parallel.

python -m paper_1712_02443_gb300.build [--force]
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libmacroaim.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXX_SRC = ["geom.cpp", "fill.cpp", "aim_setup.cpp"]
CU_SRC = ["kernels.cu", "tc_gemm.cu", "near_tc.cu", "drive.cu", "dense_gpu.cu", "fill_gpu.cu", "solver.cu", "post.cu", "capi.cu", "server.cu"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INC):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cpp", ".cu", ".cuh", ".h")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    dig = _digest()
    stamp = os.path.join(LIBDIR, "libmacroaim.sha256")
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == dig:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    cxx = os.environ.get("CXX", "g++")
    inc = ["-I", INC, "-I", CSRC]
    jobs = []
    for f in CXX_SRC:
        o = os.path.join(BUILD, f + ".o")
        jobs.append([cxx, "-O3", "-fPIC", "-std=c++17", "-pthread", "-Wall", "-Wno-sign-compare", *inc,
                     "-c", os.path.join(CSRC, f), "-o", o])
    for f in CU_SRC:
        o = os.path.join(BUILD, f + ".o")
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     *inc, "-c", os.path.join(CSRC, f), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return r

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(BUILD, f + ".o") for f in CXX_SRC + CU_SRC]
    tmp = LIB + ".tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-lcublas"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
