"""Build libhpez.so in-tree: every CUDA source compiled for sm_103a only.

The translation units compile in parallel with nvcc; the shared library is
written to ``paper_2311_12133_gb300/lib/libhpez.so``.  FMA contraction is
disabled (``-fmad=false``) on top of the explicit round-to-nearest
intrinsics the kernels use, so every binary32 operation stays one IEEE
rounding.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libhpez.so")
SOURCES = ["hpez_capi.cu", "hpez_tune.cu", "hpez_engine.cu", "hpez_sched.cu", "hpez_typed.cu",
           "k_sweep.cu",
           "k_level.cu", "k_level3d.cu", "k_level_md.cu", "k_level_md3.cu", "k_level_md3w.cu",
           "k_huffman.cu", "k_lossless.cu", "k_lorenzo.cu", "k_spline.cu",
           "k_stream.cu",
           "k_tune.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"),
              "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def flags() -> list[str]:
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
            "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
            "-Xcompiler", "-ffp-contract=off",
            "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def _deps_mtime() -> float:
    t = os.path.getmtime(os.path.join(INCLUDE, "hpez.h"))
    for f in os.listdir(CSRC):
        t = max(t, os.path.getmtime(os.path.join(CSRC, f)))
    return t


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= _deps_mtime()):
        return LIB
    cc = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *flags(), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
    # every symbol must resolve (a missing device-side definition would
    # otherwise only show when the library is loaded on the GPU machine)
    import ctypes
    ctypes.CDLL(tmp, mode=os.RTLD_NOW)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
