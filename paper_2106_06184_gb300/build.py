"""Builds libsldm.so in-tree for sm_103a (GB300) with nvcc.

Each translation unit is compiled in parallel, then linked into
``paper_2106_06184_gb300/_build/libsldm.so``.  Recompiles only what changed.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsldm.so")
SOURCES = ["mesh.cpp", "timers.cpp", "fill.cu", "fill_sub.cu", "dense.cu", "gemm_tc.cu", "lu_blocked.cu", "precond.cu",
           "mgf.cu", "nested.cu", "ports.cu", "api.cu", "serve.cpp"]
HEADERS = ["internal.h", "fill_dev.cuh", "dense.h", "gemm_tc.h", "precond.h", "mgf.h", "nested.h", os.path.join("..", "..", "include", "sldm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _flags(src):
    f = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "--expt-relaxed-constexpr"]
    if src.endswith(".cu"):
        f += ARCH
    else:
        f += ["-x", "cu"] + ARCH
    return f


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    hdr_mtime = max(os.path.getmtime(os.path.join(CSRC, h)) for h in HEADERS)
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT, s + ".o")
        if not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_mtime):
            jobs.append((src, obj))
    nvcc = _nvcc()

    def compile_one(job):
        src, obj = job
        cmd = [nvcc] + _flags(src) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(compile_one, jobs))
    objs = [os.path.join(OUT, s + ".o") for s in SOURCES]
    if jobs or not os.path.exists(LIB):
        cmd = [nvcc, "-shared"] + ARCH + objs + ["-o", LIB + ".tmp", "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
