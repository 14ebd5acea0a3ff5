"""ctypes binding of the plain C oracle (``fast_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module; the library never imports it.
It shares no code with the CUDA path.

Parity of every function here is pinned by ``tests/test_oracle_*.py`` against
closed forms, hand-built patterns, a second naive formulation and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fast_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

SAD_B, SAD_A, MT = 0, 1, 2

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no SIMD flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        ci = ctypes.c_int
        lib.oracle_abi_version.restype = ci
        lib.oracle_circle.argtypes = [ctypes.POINTER(ci), ctypes.POINTER(ci)]
        lib.oracle_halfsample.argtypes = [u8p, ci, ci, ci, u8p, ci]
        lib.oracle_arc_from_masks.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ci]
        lib.oracle_arc_from_masks.restype = ci
        lib.oracle_is_corner.argtypes = [u8p, ci, ci, ci, ci, ci]
        lib.oracle_is_corner.restype = ci
        lib.oracle_score_pixel.argtypes = [u8p, ci, ci, ci, ci, ci, ci, ci, ci]
        lib.oracle_score_pixel.restype = ci
        lib.oracle_score_map.argtypes = [u8p, ci, ci, ci, ci, ci, ci, i32p]
        lib.oracle_nms3.argtypes = [i32p, ci, ci, i32p]
        lib.oracle_nms.argtypes = [i32p, ci, ci, ci, i32p]
        lib.oracle_detect_nms.argtypes = [u8p, ci, ci, ci, ci, ci, ci, ci, ci, ci, i32p]
        lib.oracle_detect_nms.restype = ci
        lib.oracle_num_cells.argtypes = [ci, ci, ci]
        lib.oracle_num_cells.restype = ci
        lib.oracle_detect.argtypes = [u8p, ci, ci, ci, ci, ci, ci, ci, ci, i32p]
        lib.oracle_detect.restype = ci
        _lib = lib
        return lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _i32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _img(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim != 2:
        raise ValueError("expected a 2-D uint8 image")
    return img


def circle() -> list[tuple[int, int]]:
    lib = _load()
    dx = (ctypes.c_int * 16)()
    dy = (ctypes.c_int * 16)()
    lib.oracle_circle(dx, dy)
    return [(dx[i], dy[i]) for i in range(16)]


def halfsample(img: np.ndarray) -> np.ndarray:
    img = _img(img)
    h, w = img.shape
    out = np.zeros((h >> 1, w >> 1), dtype=np.uint8)
    _load().oracle_halfsample(_u8(img), w, h, w, _u8(out), w >> 1)
    return out


def pyramid(img: np.ndarray, levels: int) -> list[np.ndarray]:
    out = [_img(img)]
    for _ in range(1, levels):
        out.append(halfsample(out[-1]))
    return out


def arc_from_masks(bright: int, dark: int, n_arc: int) -> bool:
    return bool(_load().oracle_arc_from_masks(bright, dark, n_arc))


def is_corner(img: np.ndarray, x: int, y: int, t: int, n_arc: int) -> bool:
    img = _img(img)
    h, w = img.shape
    if not (3 <= x < w - 3 and 3 <= y < h - 3):
        raise ValueError("circle leaves the image")
    return bool(_load().oracle_is_corner(_u8(img), w, x, y, t, n_arc))


def score_pixel(img: np.ndarray, x: int, y: int, thresh: int, n_arc: int, mode: int = SAD_B) -> int:
    img = _img(img)
    h, w = img.shape
    return int(_load().oracle_score_pixel(_u8(img), w, h, w, x, y, thresh, n_arc, mode))


def score_map(img: np.ndarray, thresh: int, n_arc: int, mode: int = SAD_B) -> np.ndarray:
    img = _img(img)
    h, w = img.shape
    out = np.zeros((h, w), dtype=np.int32)
    _load().oracle_score_map(_u8(img), w, h, w, thresh, n_arc, mode, _i32(out))
    return out


def nms3(score: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(score, dtype=np.int32)
    h, w = s.shape
    out = np.zeros_like(s)
    _load().oracle_nms3(_i32(s), w, h, _i32(out))
    return out


def nms(score: np.ndarray, radius: int) -> np.ndarray:
    s = np.ascontiguousarray(score, dtype=np.int32)
    h, w = s.shape
    out = np.zeros_like(s)
    _load().oracle_nms(_i32(s), w, h, radius, _i32(out))
    return out


def num_cells(w: int, h: int, cell: int) -> int:
    return int(_load().oracle_num_cells(w, h, cell))


def detect(img: np.ndarray, thresh: int, n_arc: int, cell: int, levels: int,
           mode: int = SAD_B, nms_radius: int = 1) -> tuple[np.ndarray, int]:
    """Per-cell features ``(ncells, 4)`` int32 rows (x, y, level, score) and
    the number of non-empty cells; NMS over (2 nms_radius + 1)^2 windows."""
    img = _img(img)
    h, w = img.shape
    out = np.zeros((num_cells(w, h, cell), 4), dtype=np.int32)
    n = _load().oracle_detect_nms(_u8(img), w, h, w, thresh, n_arc, cell, levels, mode, nms_radius, _i32(out))
    if n < 0:
        raise MemoryError("oracle_detect: allocation failed")
    return out, int(n)
