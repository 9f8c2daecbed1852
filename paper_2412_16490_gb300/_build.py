"""Builds the in-tree CUDA library ``libbodex.so`` for sm_103a with nvcc.

The library is a plain shared object exporting the C ABI of
``include/bodex.h``; Python reaches it through ctypes (``_binding.py``).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
# translation units, compiled in parallel: the C ABI and small kernels, then
# the heavy kernel families (see bodex_kernels.cuh)
UNITS = ["bodex.cu", "qp.cu", "fused_m3.cu", "fused_m4.cu", "fused_m5.cu", "fused_multi.cu"]
SRC = [os.path.join(CSRC, u) for u in UNITS]
DEPS = SRC + [os.path.join(CSRC, "bodex_device.cuh"), os.path.join(CSRC, "bodex_kernels.cuh"),
              os.path.join(ROOT, "include", "bodex.h")]
LIB = os.path.join(HERE, "libbodex.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libbodex.so (skipped when it is newer than every source): every
    translation unit in its own nvcc process, then one link."""
    if not force and not stale():
        return LIB
    tag = f".tmp{os.getpid()}"
    objs = [os.path.join(CSRC, u[:-3] + tag + ".o") for u in UNITS]
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    procs = [subprocess.Popen([nvcc(), *flags, "-c", src, "-o", obj]) for src, obj in zip(SRC, objs)]
    codes = [p.wait() for p in procs]
    try:
        if any(codes):
            raise subprocess.CalledProcessError(next(c for c in codes if c), "nvcc -c")
        tmp = LIB + tag
        subprocess.check_call([nvcc(), *ARCH, "-shared", *objs, "-o", tmp])
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
