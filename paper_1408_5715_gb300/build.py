"""Builds the CUDA library ``_lib/libfvgb300.so`` in-tree with nvcc for sm_103a.

Translation units are compiled in parallel and linked into one shared library
with the static CUDA runtime.  No torch headers or types are involved: the
library exposes only the C ABI of ``include/fv.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libfvgb300.so")
BUILD_DIR = os.path.join(PKG, "_build")
# the bounds-checked build (-DFV_DEBUG): every table-indexed gather is tested
LIB_DEBUG = os.path.join(OUT_DIR, "libfvgb300_debug.so")
BUILD_DIR_DEBUG = os.path.join(PKG, "_build_debug")

SOURCES = ["host_mesh.cpp", "renumber.cpp", "partition.cpp", "tiles.cpp", "vertex_geom.cpp",
           "kernels.cu", "tma_step.cu",
           "tile_step.cu",
           "pair_step.cu", "closure.cu",
           "capi.cu", "totals_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(src: str, debug: bool = False):
    common = ["-O3", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
              "-Xcompiler", "-fPIC,-O2,-ffp-contract=off", "--expt-relaxed-constexpr"]
    if debug:
        common.append("-DFV_DEBUG")
    if src.endswith(".cu"):
        return common + ARCH + ["-lineinfo", "-Xptxas", "-v"]
    return common + ["-x", "c++"]


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "fv.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compiles and links the library if any source is newer; returns its path.
    debug=True builds the bounds-checked library (LIB_DEBUG) instead."""
    lib = LIB_DEBUG if debug else LIB
    build_dir = BUILD_DIR_DEBUG if debug else BUILD_DIR
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(build_dir, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        cmd = [exe, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src, debug)
        res = subprocess.run(cmd, capture_output=True, text=True)
        log = os.path.join(build_dir, src + ".log")
        with open(log, "w") as f:
            f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr[-4000:]}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [exe, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
    os.replace(tmp, lib)
    if verbose:
        for src in SOURCES:
            with open(os.path.join(build_dir, src + ".log")) as f:
                sys.stdout.write(f.read())
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                debug="--debug" in sys.argv))
