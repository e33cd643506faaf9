"""Build libipcomp.so in-tree with nvcc for sm_103a (GB300).

Each .cu unit is compiled in parallel (-gencode arch=compute_103a,code=sm_103a,
-fmad=false so that no multiply-add is contracted), then linked as a shared
library next to this file. build(bounds=True) makes the bounds-checking
variant instead (-DIPC_DEBUG_BOUNDS, libipcomp_bounds.so, its own objects):
the level kernels test every global access against its array and record the
first one outside it (ipc_debug_bounds); the binding loads it when
IPC_BOUNDS_CHECK=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libipcomp.so")
BUILD = os.path.join(HERE, "_build")
LIB_BOUNDS = os.path.join(HERE, "libipcomp_bounds.so")
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + INCLUDE, "-I" + CSRC]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src: str, bounds: bool = False) -> str:
    obj = os.path.join(BUILD_BOUNDS if bounds else BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC] + ARCH + FLAGS + (["-DIPC_DEBUG_BOUNDS"] if bounds else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    lib = LIB_BOUNDS if bounds else LIB
    if not force and up_to_date(lib):
        return lib
    os.makedirs(BUILD_BOUNDS if bounds else BUILD, exist_ok=True)
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, bounds), srcs))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        print("built", lib, file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, bounds="--bounds" in sys.argv)
