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
# the checked build: every index check of the device code enabled (-DVIO_CHECKED)
CHECKED_LIB_PATH = os.path.join(OUT_DIR, "libvio_gb300_checked.so")

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


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles the library when a source is newer than it; returns its path.
    Translation units compile in parallel, then one link step.  checked=True
    builds the variant with the device-side index checks enabled."""
    from concurrent.futures import ThreadPoolExecutor

    os.makedirs(OUT_DIR, exist_ok=True)
    lib_path = CHECKED_LIB_PATH if checked else LIB_PATH
    if not force and os.path.exists(lib_path):
        t = os.path.getmtime(lib_path)
        if all(os.path.getmtime(p) <= t for p in _deps()):
            return lib_path
    pid = os.getpid()
    tag = "chk." if checked else ""
    objs = [os.path.join(OUT_DIR, os.path.basename(src) + f".{tag}{pid}.o") for src in _sources()]
    extra = ["-DVIO_CHECKED"] if checked else []

    def compile_one(args):
        src, obj = args
        cmd = [nvcc(), *NVCC_FLAGS, *extra, "-c", "-I", INCLUDE, "-o", obj, src]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)

    tmp = lib_path + f".tmp{pid}"
    try:
        with ThreadPoolExecutor(max(1, len(objs))) as ex:
            list(ex.map(compile_one, zip(_sources(), objs)))
        link = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(link))
        subprocess.check_call(link)
        os.replace(tmp, lib_path)
    finally:
        for o in objs + [tmp]:
            if os.path.exists(o):
                os.remove(o)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
