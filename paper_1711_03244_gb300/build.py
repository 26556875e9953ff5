"""Builds the CUDA library in-tree for sm_103a (GB300): libmcx_gb300.so next to this file.

Each translation unit is compiled by its own nvcc process in parallel, then linked into one
shared library against the shared CUDA runtime.  No CMake, no JIT.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmcx_gb300.so")
SOURCES = ["walk.cu", "api.cu", "noalloc.cu", "batch.cu", "denoise.cu", "probe.cu"]
HEADERS = ["mcx_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")

# Single-precision math: flush denormals, approximate division and square root (the hot
# path calls the hardware intrinsics explicitly; these flags govern the remaining float
# operators).  FP64 code is unaffected.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-ftz=true",
              "-prec-div=false", "-prec-sqrt=false", "-Xptxas", "-v"] + ARCH


def _nvcc() -> str:
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(HERE, "..", "include", "mcx.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, log: list) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj,
           "-I", os.path.join(HERE, "..", "include")] + NVCC_FLAGS
    r = subprocess.run(cmd, capture_output=True, text=True)
    log.append((src, r.stdout + r.stderr))
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links the library if any source is newer than it; returns its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    log: list = []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, log), SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + [
        "-cudart", "shared", "-Xlinker", "-rpath", "-Xlinker", os.path.join(CUDA_HOME, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for src, text in log:
            f.write(f"== {src}\n{text}\n")
    if verbose:
        for src, text in log:
            print(f"== {src}\n{text}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
