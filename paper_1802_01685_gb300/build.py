"""Builds libbf.so (the CUDA library behind include/bf.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into a
shared library with the CUDA runtime linked statically, so loading it needs no
CUDA driver (the C-ABI symbol check runs on machines without a GPU).

build(debug_bounds=True) makes libbf_debug.so instead: the same library with
-DBF_DEBUG_BOUNDS, whose kernels check the indices they rely on (recording a
code in the context's status word rather than trapping) and whose result
buffers carry canaries checked after each search.  Loading it: set
BF_LIBRARY to its path before importing the binding.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbf.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(PKG, "libbf_debug.so")

SOURCES = ["api.cu", "serve.cu", "bank.cu", "prep.cu", "corr_simt.cu", "corr_tc.cu",
           "finalize.cu", "permute.cu", "noalloc.cu", "plan.cu", "predict.cu", "corr_fft.cu", "probe.cu"]
HEADERS = ["bf_internal.h", "runtime.h", "corr_common.cuh", "synth.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# hidden visibility: only the declarations of include/bf.h are exported
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-Wall", "-Xcompiler", "-fvisibility=hidden",
                     "-DBF_BUILDING_LIBRARY", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "bf.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, verbose: bool, build_dir: str = BUILD, extra=()) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc()] + NVCC_FLAGS + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    """Compile and link libbf.so (libbf_debug.so with debug_bounds) unless it
    is newer than every input."""
    lib, build_dir = (LIB_DEBUG, BUILD_DEBUG) if debug_bounds else (LIB, BUILD)
    extra = ["-DBF_DEBUG_BOUNDS"] if debug_bounds else []
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(build_dir, exist_ok=True)
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, build_dir, extra), SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs + [
        "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                debug_bounds="--debug-bounds" in sys.argv))
