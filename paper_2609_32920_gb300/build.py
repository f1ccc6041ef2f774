"""Build liblt.so in-tree with nvcc for sm_103a (GB300).  No torch extension machinery:
the library exposes a plain C ABI (include/lt.h)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "liblt.so")
BUILD = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress", "177"]
# (source, object, extra flags): the kernels are compiled once per BVH width.  They are
# compiled without multiply-add contraction: every pass of a method replays the same path
# and must take the same discrete decisions (a ray through a shared triangle edge, a
# connection at the film border), but the compiler would otherwise fuse the same source
# expression differently in each kernel it is inlined into.  Explicit fmaf() calls stay fused.
KERNEL_FLAGS = ["-fmad=false"]
UNITS = [("lt_api.cu", "lt_api.o", []), ("lt_dispatch.cu", "lt_dispatch.o", []), ("lt_mlp.cu", "lt_mlp.o", []),
         ("lt_kernels.cu", "lt_kernels_w2.o", ["-DLT_BVH_WIDTH=2", *KERNEL_FLAGS]),
         ("lt_kernels.cu", "lt_kernels_w4.o", ["-DLT_BVH_WIDTH=4", *KERNEL_FLAGS]),
         ("lt_kernels.cu", "lt_kernels_w8.o", ["-DLT_BVH_WIDTH=8", *KERNEL_FLAGS])]
SOURCES = sorted({u[0] for u in UNITS})


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "lt.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(unit):
        src, obj, extra = unit
        obj = os.path.join(BUILD, obj)
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = OUT + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
