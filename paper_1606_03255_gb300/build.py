"""Build libfl.so (the CUDA library behind include/fl.h) for sm_103a, in-tree.

Each translation unit under csrc/ is compiled by nvcc in parallel and the
objects are linked into ``_build/libfl.so``.  No torch extension machinery is
involved: the library exposes a plain C ABI.  ``peaks/fl_peaks.cu`` becomes
``_build/libflpeaks.so``, the FMA-rate microbenchmark the benchmark reads its
FP32/FP64 pipe peaks from (measurement only, not part of the C ABI).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfl.so")
PEAKS_SRC = os.path.join(HERE, "peaks", "fl_peaks.cu")
PEAKS_LIB = os.path.join(BUILD, "libflpeaks.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INC, "-I", SRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile csrc/*.cu and link libfl.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(SRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(SRC, "*.cuh")) + glob.glob(os.path.join(INC, "*.h")))
    cc = nvcc()
    extra = list(extra or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src, *headers]):
            cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            subprocess.run(cmd, check=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources))
    if force or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    if force or _stale(PEAKS_LIB, [PEAKS_SRC]):
        tmp = PEAKS_LIB + f".{os.getpid()}.tmp"
        subprocess.run([cc, *ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", PEAKS_SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, PEAKS_LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
