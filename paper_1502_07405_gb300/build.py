"""Build the sm_103a shared library libhssmf.so in-tree (nvcc, no cmake).

Each translation unit is compiled in parallel, then linked with -shared.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhssmf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["analyze.cpp", "k_dense.cu", "k_solve.cu", "k_hss.cu", "k_id_rx.cu", "k_gemm_tc.cu", "k_gemm_tma.cu", "hss.cu", "solver.cu", "noalloc.cu"]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhssmf")
    return p


def _compile(src, extra):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    cmd = [_nvcc(), "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH,
           "-I", CSRC, "-I", os.path.join(HERE, "..", "include"), "-c", os.path.join(CSRC, src),
           "-o", obj, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, extra=()):
    os.makedirs(OUT_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log.strip():
                print(log)
    cmd = [_nvcc(), "-shared", *ARCH, "-o", LIB, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
