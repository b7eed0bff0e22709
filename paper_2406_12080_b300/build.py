"""Build libh3dgs.so in-tree with nvcc for sm_103a (B300).

Usage: python -m paper_2406_12080_b300.build [--force] [--verbose] [--check]
The shared library links the CUDA runtime statically, so it loads (and reports
H3DGS_ERR_NO_DEVICE) on machines without a GPU.
"""
from __future__ import annotations

import argparse
import fcntl
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libh3dgs.so")
BUILD_DIR = os.path.join(PKG, "_build")
# the debug build with bounds checks in the kernels (-DH3DGS_CHECK; see h3dgs_build_flags in h3dgs.h)
LIB_CHECK = os.path.join(PKG, "libh3dgs_check.so")
BUILD_DIR_CHECK = os.path.join(PKG, "_build", "check")

SOURCES = ["api.cu", "cut.cu", "preprocess.cu", "sort.cu", "blend.cu", "backward.cu", "builder.cu", "cut_noalloc.cu", "compact.cu", "stream.cu", "calib.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "h3dgs.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, check: bool = False) -> str:
    """Compile libh3dgs.so (check=True: libh3dgs_check.so, the bounds-checked debug build)."""
    lib, bdir = (LIB_CHECK, BUILD_DIR_CHECK) if check else (LIB, BUILD_DIR)
    if not force and not _stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    # one build at a time per build folder (every rank of a multi-GPU run calls this): a caller that
    # waited for the lock finds the library fresh and returns
    with open(os.path.join(bdir, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        if not force and not _stale(lib):
            return lib
        return _compile(lib, bdir, check, verbose, ptxas_verbose)


def _compile(lib: str, bdir: str, check: bool, verbose: bool, ptxas_verbose: bool) -> str:
    extra = (["-Xptxas", "-v"] if ptxas_verbose else []) + (["-DH3DGS_CHECK"] if check else [])
    objs = [os.path.join(bdir, src.replace(".cu", ".o")) for src in SOURCES]
    cmds = [[nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj] for src, obj in zip(SOURCES, objs)]
    if verbose:
        for cmd in cmds:
            print(" ".join(cmd), flush=True)
    # translation units compile independently: run them side by side
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
        list(ex.map(subprocess.check_call, cmds))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-verbose", action="store_true")
    ap.add_argument("--check", action="store_true", help="the bounds-checked debug build (libh3dgs_check.so)")
    a = ap.parse_args()
    print(build(a.force, a.verbose, a.ptxas_verbose, a.check))
    sys.exit(0)
