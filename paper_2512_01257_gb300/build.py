"""Build librafeast.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked into
``paper_2512_01257_gb300/librafeast.so`` against the shared CUDA runtime.

    python -m paper_2512_01257_gb300.build [--verbose] [NVCC_FLAG ...]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librafeast.so")
SOURCES = ["kernels_sparse.cu", "kernels_batched.cu", "kernels_tma.cu", "kernels_dense.cu",
           "kernels_tiled.cu", "kernels_tc.cu", "api.cu", "noalloc.cu", "hostmath.cpp", "tiling.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, extra, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O3", "-Xcompiler", "-pthread", "-I", os.path.join(os.path.dirname(PKG), "include"),
           "--diag-suppress", "177", "-c", os.path.join(CSRC, src), "-o", obj, *extra]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "c++")
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr.strip():
        print(res.stderr, flush=True)
    return obj


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra), verbose), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xcompiler", "-pthread", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser(
        epilog="Any other argument (e.g. -DNAME=VALUE) is passed to nvcc for every unit.")
    ap.add_argument("--verbose", action="store_true")
    a, extra = ap.parse_known_args(argv)
    print(build(a.verbose, extra))


if __name__ == "__main__":
    main(sys.argv[1:])
