"""Builds the CUDA library in-tree: ``_build/libvio_gb300.so`` for sm_103a."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libvio_gb300.so")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
]


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + \
        sorted(glob.glob(os.path.join(INCLUDE, "*.h")))


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the library when a source is newer than it; returns its path.
    Translation units compile in parallel, then one link step."""
    from concurrent.futures import ThreadPoolExecutor

    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(p) <= t for p in _deps()):
            return LIB_PATH
    pid = os.getpid()
    objs = [os.path.join(OUT_DIR, os.path.basename(src) + f".{pid}.o") for src in _sources()]

    def compile_one(args):
        src, obj = args
        cmd = [nvcc(), *NVCC_FLAGS, "-c", "-I", INCLUDE, "-o", obj, src]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)

    tmp = LIB_PATH + f".tmp{pid}"
    try:
        with ThreadPoolExecutor(max(1, len(objs))) as ex:
            list(ex.map(compile_one, zip(_sources(), objs)))
        link = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(link))
        subprocess.check_call(link)
        os.replace(tmp, LIB_PATH)
    finally:
        for o in objs + [tmp]:
            if os.path.exists(o):
                os.remove(o)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
