"""Builds libsaa.so (the C-ABI CUDA library) in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled by nvcc in parallel, then
linked into ``_build/libsaa.so``.  Rebuilds only what changed.  The
index-checked variant (SAA_BOUNDS_CHECK defined: kernels report an index
past its buffer in the error word instead of faulting) builds the same way
into ``_build/bounds/`` and ``_build/libsaa_bounds.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsaa.so")
LIB_BOUNDS = os.path.join(BUILD, "libsaa_bounds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
           "--expt-relaxed-constexpr", f"-I{os.path.join(ROOT, 'include')}"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: libsaa needs the CUDA 13 toolkit to build")
    return p


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "saa.h")]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, extra: list[str], objdir: str = BUILD) -> str:
    obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _deps_mtime()):
        return obj
    tmp = obj + f".{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, *NVFLAGS, *extra, "-c", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, obj)
    return obj


def build(verbose: bool = False, extra: list[str] | None = None, bounds: bool = False) -> str:
    """Compiles every csrc/*.cu and links _build/libsaa.so (with bounds=True:
    the index-checked _build/libsaa_bounds.so); returns its path."""
    objdir = os.path.join(BUILD, "bounds") if bounds else BUILD
    lib = LIB_BOUNDS if bounds else LIB
    os.makedirs(objdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = list(extra or []) + (["-DSAA_BOUNDS_CHECK"] if bounds else [])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, objdir), srcs))
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose:
        print(lib)
    return lib


def ptxas_report(src: str) -> str:
    """-Xptxas -v register / spill / shared-memory report of one source."""
    cmd = [nvcc(), *ARCH, *NVFLAGS, "-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.stdout + r.stderr


if __name__ == "__main__":
    build(verbose=True)
