"""Compile the qbvh CUDA sources into the in-tree shared library ``libqbvh.so``.

nvcc compiles every translation unit for sm_103a only, in parallel, then links
them with the static CUDA runtime so that the library has no dependency
beyond the driver.  Re-running is cheap: units are rebuilt only when a source
or header is newer than their object file.

Usage:  python -m paper_1901_08088_gb300.build_lib [--force] [--verbose]
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqbvh.so")
HEADERS = [os.path.join(CSRC, "qbvh_internal.cuh"), os.path.join(ROOT, "include", "qbvh.h")]
SOURCES = ["api.cu", "build.cu", "sort.cu", "query.cu", "lj.cu", "noalloc.cu", "grid.cu", "small_build.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fsigned-char",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the qbvh library needs the CUDA toolkit to build")
    return exe


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, force: bool, verbose: bool, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if force or _stale(obj, [path, *HEADERS]):
        cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, flush=True)
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Build libqbvh.so.  Extra nvcc flags (tuning macros such as
    -DQBVH_LEAF_BATCH=8) come from `extra` or the QBVH_NVCC_FLAGS variable;
    changing them forces a rebuild."""
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or []) + os.environ.get("QBVH_NVCC_FLAGS", "").split()
    stamp = os.path.join(BUILD, "flags.txt")
    flags_now = " ".join(extra)
    if not os.path.exists(stamp) or open(stamp).read() != flags_now:
        force = True
        with open(stamp, "w") as fh:
            fh.write(flags_now)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, verbose, extra), SOURCES))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    args = sys.argv[1:]
    extra = [a[len("--xptxas="):] for a in args if a.startswith("--xptxas=")]
    build(force="--force" in args, verbose="--verbose" in args,
          extra=(["-Xptxas", "-v"] if "--ptxas-v" in args else []))
    print(LIB)
