"""Compiles the CUDA library ``libgjp.so`` in-tree for sm_103a with nvcc.

    python -m paper_1609_00958_gb300.build
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("gjp.cu", "gjp_batch.cu", "gjp_texture.cu")]
LIB = os.path.join(HERE, "libgjp.so")
# debug build: every tap of the unchecked interior marches range-checked (GJP_CHECK_TAPS)
LIB_CHECKED = os.path.join(HERE, "libgjp_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libgjp.so")
    return cand


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = SOURCES + [os.path.join(INCLUDE, "gjp.h")] + [
        os.path.join(HERE, "csrc", f) for f in os.listdir(os.path.join(HERE, "csrc"))]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=None, lib: str = LIB) -> str:
    """Compiles every translation unit in parallel (one nvcc each), then
    links the shared library `lib`; returns its path."""
    if not force and not stale(lib):
        return lib
    tag = f".{os.path.basename(lib)}.{os.getpid()}.tmp"   # objects: <name>.<lib>.<pid>.tmp.o (nvcc reads the suffix)
    flags = [*(extra or []), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    objs = [os.path.splitext(src)[0] + tag + ".o" for src in SOURCES]
    procs = [subprocess.Popen([nvcc(), *flags, "-c", src, "-o", obj]) for src, obj in zip(SOURCES, objs)]
    codes = [p.wait() for p in procs]
    try:
        for src, code in zip(SOURCES, codes):
            if code != 0:
                raise subprocess.CalledProcessError(code, f"nvcc -c {src}")
        tmp = lib + tag
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.unlink(obj)
    return lib


def build_checked(force: bool = False) -> str:
    """The debug library: the same sources with GJP_CHECK_TAPS=1."""
    return build(force=force, extra=["-DGJP_CHECK_TAPS=1"], lib=LIB_CHECKED)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
