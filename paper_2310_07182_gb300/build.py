"""Build libcr.so in-tree with nvcc for sm_103a (translation units compiled in parallel)."""
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
LIB = os.path.join(PKG, "libcr.so")
# the debug build: every node, triangle and material index checked in the kernels (CR_DEBUG=1)
LIB_DEBUG = os.path.join(PKG, "libcr_debug.so")
SOURCES = ["trace.cu", "trace_bvh8.cu", "path.cu", "cr_api.cpp", "bvh_build.cpp", "bvh8_build.cpp", "trace_static.cu", "server.cpp", "probe.cu", "trace_bvh4.cu", "bvh4_build.cpp"]
HEADERS = ["cr_internal.h", "device_math.cuh", "trace_common.cuh", "debug_checks.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(src: str):
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if src.endswith(".cu"):
        return common + ARCH + ["-lineinfo", "-Xptxas", "-O3"]
    return common + ["-Xcompiler", "-O2", "-Xcompiler", "-ffp-contract=off"]


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "cr.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    build_dir = BUILD + ("_debug" if debug else "")
    if debug:
        extra_flags = list(extra_flags) + ["-DCR_DEBUG=1"]
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(build_dir, exist_ok=True)
    nv = nvcc()

    def compile_one(src):
        obj = os.path.join(build_dir, src + ".o")
        cmd = [nv, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src) + list(extra_flags)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nv, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-pthread", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [], debug="--debug" in sys.argv))
