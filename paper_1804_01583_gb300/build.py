"""Build libkv.so (the CUDA library behind include/kv.h) for sm_103a.

Each .cu translation unit is compiled by its own nvcc process in parallel,
then linked into paper_1804_01583_gb300/_build/libkv.so.  No CMake; the only
requirement is nvcc from CUDA 13 on PATH or in /usr/local/cuda/bin.
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
LIB = os.path.join(BUILD, "libkv.so")
# the debug build (-DKV_DEBUG: device-side index checks on the matrix and the
# scattered columns, a test hook), in a directory of its own
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
SOURCES = ["kv_abi.cu", "k_stencil.cu", "k_vector.cu", "k_expm.cu", "k_bounds.cu", "k_csr.cu", "k_stencil_tma.cu", "k_stencil_tma64.cu",
           "k_noalloc.cu", "kv_serve.cu", "kv_graph.cu", "k_lognorm.cu",
           "k_expm_large.cu", "k_csr_transpose.cu", "k_csr_check.cu", "k_lp.cu", "k_diag.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-diag-suppress", "177"]


def nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libkv")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "kv.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files if os.path.exists(f))


def build(force: bool = False, verbose: bool = False, extra: list | None = None, debug: bool = False) -> str:
    bdir = BUILD_DEBUG if debug else BUILD
    lib = os.path.join(bdir, "libkv.so")
    os.makedirs(bdir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    cc = nvcc()
    extra = list(extra or []) + (["-DKV_DEBUG"] if debug else [])

    def compile_one(src: str) -> str:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
