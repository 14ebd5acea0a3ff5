"""Thin ctypes binding of ``include/vio.h``.

Argument marshalling only: every step of the detector runs in the CUDA
library.  PyTorch provides device memory (``tensor.data_ptr()``) and streams
(``torch.cuda.Stream.cuda_stream``).  Loading fails loudly when the library
has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

SCORE_SAD_B, SCORE_SAD_A, SCORE_MT = 0, 1, 2
MAX_LEVELS = 5

STATUS = {0: "VIO_OK", 1: "VIO_ERR_INVALID_ARG", 2: "VIO_ERR_OOM", 3: "VIO_ERR_CUDA",
          4: "VIO_ERR_TIMEOUT", 5: "VIO_ERR_BUSY", 6: "VIO_ERR_UNSUPPORTED", 7: "VIO_ERR_NOT_FOUND"}


class VioError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("max_frames", ctypes.c_int), ("score", ctypes.c_int),
                ("autotune", ctypes.c_int), ("use_graphs", ctypes.c_int), ("profile", ctypes.c_int),
                ("nms_radius", ctypes.c_int)]


class Dims(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("pitch", ctypes.c_int32)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("thresh", ctypes.c_int), ("arc_len", ctypes.c_int), ("cell_size", ctypes.c_int),
                ("levels", ctypes.c_int), ("max_batch", ctypes.c_int), ("max_wait_us", ctypes.c_int),
                ("lanes", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("queue_capacity", ctypes.c_int), ("keep_results", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("frames_per_s", ctypes.c_double), ("max_batch_frames", ctypes.c_uint64),
                ("max_lanes_in_flight", ctypes.c_uint64), ("overlapped_batches", ctypes.c_uint64)]


class TrackParams(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("patch_fine", ctypes.c_int), ("patch_coarse", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("min_update", ctypes.c_float), ("model", ctypes.c_int)]


TRACK_GAIN, TRACK_OFFSET = 1, 2
TRACK_RESULT_WORDS = 8  # x, y, gain, offset (float) | status, iters (int32) | residual (float) | reserved


class Tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int),
                ("cta_per_sm", ctypes.c_int), ("variant", ctypes.c_int), ("nms_radius", ctypes.c_int),
                ("cell_size", ctypes.c_int)]


_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/vio.h."""
    with open(os.path.join(_build.INCLUDE, "vio.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vio_[a-z0-9_]+)\s*\(", text)))


def lib_path() -> str:
    """Path of the library load() uses (the checked build with VIO_CHECKED=1)."""
    return _build.CHECKED_LIB_PATH if os.environ.get("VIO_CHECKED") == "1" else _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Loads the library (building it first if asked and needed).  With
    VIO_CHECKED=1 in the environment the checked build (device-side index
    checks enabled) is loaded instead."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("VIO_CHECKED") == "1"
    path = lib_path()
    if build_if_missing:
        path = _build.build(checked=checked)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    ci = ctypes.c_int
    st = ctypes.c_int
    lib.vio_config_default.argtypes = [ctypes.POINTER(Config)]
    lib.vio_config_default.restype = None
    lib.vio_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Config)]
    lib.vio_create.restype = st
    lib.vio_destroy.argtypes = [P]
    lib.vio_destroy.restype = st
    lib.vio_status_str.argtypes = [st]
    lib.vio_status_str.restype = ctypes.c_char_p
    lib.vio_last_error.argtypes = [P]
    lib.vio_last_error.restype = ctypes.c_char_p
    lib.vio_num_cells.argtypes = [ci, ci, ci]
    lib.vio_num_cells.restype = ctypes.c_size_t
    detect_args = [P, ctypes.POINTER(P), ctypes.POINTER(Dims), ci, ci, ci, ci, ci, ctypes.POINTER(P), P, P]
    lib.vio_detect.argtypes = detect_args
    lib.vio_detect.restype = st
    lib.vio_detect_host.argtypes = detect_args
    lib.vio_detect_host.restype = st
    lib.vio_detect_host_async.argtypes = detect_args
    lib.vio_detect_host_async.restype = st
    lib.vio_detect_sweep.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(Dims), ci, ctypes.POINTER(ci),
                                     ctypes.POINTER(ci), ci, ci, ci, ctypes.POINTER(P), P, P]
    lib.vio_detect_sweep.restype = st
    lib.vio_sync.argtypes = [P, P]
    lib.vio_sync.restype = st
    lib.vio_selftest_timeout.argtypes = [P, ctypes.c_uint32]
    lib.vio_selftest_timeout.restype = st
    lib.vio_stage_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.vio_stage_ms.restype = st
    lib.vio_get_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    lib.vio_get_tuning.restype = st
    lib.vio_set_tuning.argtypes = [P, ctypes.POINTER(Tuning)]
    lib.vio_set_tuning.restype = st
    lib.vio_device.argtypes = [P]
    lib.vio_device.restype = ci
    lib.vio_get_config.argtypes = [P, ctypes.POINTER(Config)]
    lib.vio_get_config.restype = st
    lib.vio_track_params_default.argtypes = [ctypes.POINTER(TrackParams)]
    lib.vio_track_params_default.restype = None
    lib.vio_track.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(Dims), ci, ctypes.POINTER(P),
                              ctypes.POINTER(ci), ctypes.POINTER(TrackParams), ctypes.POINTER(P), P]
    lib.vio_track.restype = st
    lib.vio_track_cells.argtypes = lib.vio_track.argtypes
    lib.vio_track_cells.restype = st
    lib.vio_serve_config_default.argtypes = [ctypes.POINTER(ServeConfig)]
    lib.vio_serve_config_default.restype = None
    lib.vio_serve_start.argtypes = [P, ctypes.POINTER(ServeConfig)]
    lib.vio_serve_start.restype = st
    lib.vio_submit.argtypes = [P, ci, P, Dims, ctypes.POINTER(ctypes.c_uint64)]
    lib.vio_submit.restype = st
    lib.vio_poll.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ci)]
    lib.vio_poll.restype = st
    lib.vio_serve_drain.argtypes = [P, ci]
    lib.vio_serve_drain.restype = st
    lib.vio_serve_stats.argtypes = [P, ctypes.POINTER(ServeStats)]
    lib.vio_serve_stats.restype = st
    lib.vio_serve_stop.argtypes = [P]
    lib.vio_serve_stop.restype = st
    lib.vio_detect_noalloc.argtypes = [P, Dims, ci, ci, ci, ci, ci, P, P, P]
    lib.vio_detect_noalloc.restype = st
    lib.vio_autotune_log.argtypes = [P, ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_float), ci]
    lib.vio_autotune_log.restype = ci
    lib.vio_copy_level.argtypes = [P, ci, ci, P, ci, P]
    lib.vio_copy_level.restype = st
    lib.vio_num_variants.argtypes = []
    lib.vio_num_variants.restype = ci
    lib.vio_variant.argtypes = [ci, ctypes.POINTER(Tuning)]
    lib.vio_variant.restype = st
    _lib = lib
    return lib


def num_cells(w: int, h: int, cell: int) -> int:
    return int(load().vio_num_cells(w, h, cell))


def variants() -> list[tuple[int, int, int]]:
    """(tile_w, tile_h, nms_radius) of every built variant, by variant index."""
    lib = load()
    out = []
    for i in range(lib.vio_num_variants()):
        t = Tuning()
        lib.vio_variant(i, ctypes.byref(t))
        out.append((t.tile_w, t.tile_h, t.nms_radius))
    return out


def track_fields(res):
    """Splits (n, 8) float32 tracker records (numpy) into
    (xy float32 (n, 2), gain, offset, status int32, iters int32, residual)."""
    import numpy as np

    r = np.ascontiguousarray(res, dtype=np.float32)
    ints = r.view(np.int32)
    return r[:, 0:2], r[:, 2], r[:, 3], ints[:, 4], ints[:, 5], r[:, 6]


def variant_ids(nms_radius: int = 1) -> list[int]:
    """Indices of the variants built for one NMS radius."""
    return [i for i, v in enumerate(variants()) if v[2] == nms_radius]


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    h = getattr(stream, "cuda_stream", stream)
    return ctypes.c_void_p(int(h) if h else 0)


class HostBatch:
    """Host frames and result buffers marshalled once for repeated
    vio_detect_host / vio_detect_host_async calls on the same buffers (a
    camera ring's fixed slots): frames are 2-D uint8 numpy arrays, outs numpy
    int32 (n_cells, 4) arrays (pinned for the asynchronous call), counts an
    int32 array or None.  The caller rewrites the buffers' contents between
    calls; the arrays must stay alive while the batch is used."""

    def __init__(self, frames, outs, counts=None):
        n = len(frames)
        if len(outs) != n:
            raise ValueError("one output array per frame")
        self.n = n
        self.dims = (Dims * n)()
        self.fptr = (ctypes.c_void_p * n)()
        for i, f in enumerate(frames):
            if f.dtype != np.uint8 or f.ndim != 2 or f.strides[1] != 1:
                raise ValueError("frames must be 2-D uint8 arrays with unit column stride")
            self.dims[i] = Dims(f.shape[1], f.shape[0], f.strides[0])
            self.fptr[i] = f.ctypes.data
        self.optr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
        self.cptr = ctypes.c_void_p(counts.ctypes.data) if counts is not None else None
        self._keep = (frames, outs, counts)


class Detector:
    """One library context on one device."""

    def __init__(self, device: int = 0, max_frames: int = 64, score: int = SCORE_SAD_B,
                 mem_budget_bytes: int = 0, autotune: bool = False, use_graphs: bool = True,
                 profile: bool = False, nms_radius: int = 1):
        self.lib = load()
        cfg = Config()
        self.lib.vio_config_default(ctypes.byref(cfg))
        cfg.device = device
        cfg.max_frames = max_frames
        cfg.score = score
        cfg.mem_budget_bytes = mem_budget_bytes
        cfg.autotune = int(autotune)
        cfg.use_graphs = int(use_graphs)
        cfg.profile = int(profile)
        cfg.nms_radius = nms_radius
        self.cfg = cfg
        self.ctx = ctypes.c_void_p()
        s = self.lib.vio_create(ctypes.byref(self.ctx), ctypes.byref(cfg))
        if s != 0:
            raise VioError(s, self.lib.vio_status_str(s).decode())

    def close(self):
        if self.ctx:
            self.lib.vio_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s: int):
        if s != 0:
            raise VioError(s, self.lib.vio_last_error(self.ctx).decode())

    def detect(self, frames, thresh: int, arc_len: int, cell: int, levels: int,
               outs=None, counts=None, stream=None):
        """frames: list of 2-D uint8 CUDA tensors (row stride = pitch).
        Returns (list of (ncells, 4) int32 CUDA tensors, int32 counts tensor)."""
        import torch

        n = len(frames)
        dims = (Dims * n)()
        fptr = (ctypes.c_void_p * n)()
        for i, f in enumerate(frames):
            if f.dtype != torch.uint8 or f.dim() != 2 or f.stride(1) != 1 or not f.is_cuda:
                raise ValueError("frames must be 2-D uint8 CUDA tensors with unit column stride")
            dims[i] = Dims(f.shape[1], f.shape[0], f.stride(0))
            fptr[i] = f.data_ptr()
        dev = frames[0].device
        if outs is None:
            outs = [torch.empty((num_cells(d.w, d.h, cell or 32), 4), dtype=torch.int32, device=dev) for d in dims]
        if counts is None:
            counts = torch.empty(n, dtype=torch.int32, device=dev)
        optr = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        self._check(self.lib.vio_detect(self.ctx, fptr, dims, n, thresh, arc_len, cell, levels, optr,
                                        ctypes.c_void_p(counts.data_ptr()), _stream_handle(stream)))
        self._last_dims = [(d.w, d.h) for d in dims]
        return outs, counts

    def track(self, prev, nxt, pts, params: dict | None = None, outs=None, stream=None):
        """Feature tracking (Section II-E) of pts[i] from prev[i] to nxt[i].

        prev, nxt: lists of 2-D uint8 CUDA tensors (same size per pair);
        pts: list of (n_i, 2) float32 CUDA tensors of level-0 (x, y);
        params: overrides of vio_track_params fields.  Returns a list of
        (n_i, 8) float32 CUDA tensors in the vio_track_result layout (use
        track_fields to split them)."""
        import torch

        n = len(prev)
        if len(nxt) != n or len(pts) != n:
            raise ValueError("prev, nxt and pts must have one entry per pair")
        dims = (Dims * n)()
        pp = (ctypes.c_void_p * n)()
        nn = (ctypes.c_void_p * n)()
        for i, (a, b) in enumerate(zip(prev, nxt)):
            for f in (a, b):
                if f.dtype != torch.uint8 or f.dim() != 2 or f.stride(1) != 1 or not f.is_cuda:
                    raise ValueError("frames must be 2-D uint8 CUDA tensors with unit column stride")
            if a.shape != b.shape or a.stride(0) != b.stride(0):
                raise ValueError("both frames of a pair need the same size and pitch")
            dims[i] = Dims(a.shape[1], a.shape[0], a.stride(0))
            pp[i] = a.data_ptr()
            nn[i] = b.data_ptr()
        for q in pts:
            if q.dtype != torch.float32 or q.dim() != 2 or q.shape[1] != 2 or not q.is_contiguous():
                raise ValueError("pts must be contiguous (n, 2) float32 tensors")
        if outs is None:
            outs = [torch.empty((q.shape[0], TRACK_RESULT_WORDS), dtype=torch.float32, device=q.device) for q in pts]
        tp = TrackParams()
        self.lib.vio_track_params_default(ctypes.byref(tp))
        for k, v in (params or {}).items():
            setattr(tp, k, v)
        qp = (ctypes.c_void_p * n)(*[q.data_ptr() for q in pts])
        cnt = (ctypes.c_int * n)(*[q.shape[0] for q in pts])
        op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        self._check(self.lib.vio_track(self.ctx, pp, nn, dims, n, qp, cnt, ctypes.byref(tp), op,
                                       _stream_handle(stream)))
        return outs

    def track_cells(self, prev, nxt, cells, params: dict | None = None, outs=None, stream=None):
        """Tracks the detector's records: cells[i] is the (ncells, 4) int32
        CUDA tensor a detection of prev[i] returned; one (ncells, 8) result
        per cell (empty cells give status 0)."""
        import torch

        n = len(prev)
        if len(nxt) != n or len(cells) != n:
            raise ValueError("prev, nxt and cells must have one entry per pair")
        dims = (Dims * n)()
        pp = (ctypes.c_void_p * n)()
        nn = (ctypes.c_void_p * n)()
        for i, (a, b) in enumerate(zip(prev, nxt)):
            if a.shape != b.shape or a.stride(0) != b.stride(0) or a.dtype != torch.uint8 or not a.is_cuda:
                raise ValueError("both frames of a pair need the same size and pitch (uint8 CUDA tensors)")
            dims[i] = Dims(a.shape[1], a.shape[0], a.stride(0))
            pp[i] = a.data_ptr()
            nn[i] = b.data_ptr()
        for c in cells:
            if c.dtype != torch.int32 or c.dim() != 2 or c.shape[1] != 4 or not c.is_contiguous():
                raise ValueError("cells must be contiguous (n, 4) int32 tensors")
        if outs is None:
            outs = [torch.empty((c.shape[0], TRACK_RESULT_WORDS), dtype=torch.float32, device=c.device) for c in cells]
        tp = TrackParams()
        self.lib.vio_track_params_default(ctypes.byref(tp))
        for k, v in (params or {}).items():
            setattr(tp, k, v)
        cp = (ctypes.c_void_p * n)(*[c.data_ptr() for c in cells])
        cnt = (ctypes.c_int * n)(*[c.shape[0] for c in cells])
        op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        self._check(self.lib.vio_track_cells(self.ctx, pp, nn, dims, n, cp, cnt, ctypes.byref(tp), op,
                                             _stream_handle(stream)))
        return outs

    def track_cells_ptrs(self, pp, nn, dims, n, cp, cnt, tp, op, stream_handle):
        """Pre-marshalled vio_track_cells call (ctypes arrays), for timing loops."""
        self._check(self.lib.vio_track_cells(self.ctx, pp, nn, dims, n, cp, cnt, ctypes.byref(tp), op,
                                             stream_handle))

    def detect_sweep(self, frames, params, cell: int, levels: int, stream=None):
        """params: list of (thresh, arc_len).  Returns (outs[p][i] tensors, counts (n_params, n))."""
        import torch

        n, npar = len(frames), len(params)
        dims = (Dims * n)()
        fptr = (ctypes.c_void_p * n)()
        for i, f in enumerate(frames):
            if f.dtype != torch.uint8 or f.dim() != 2 or f.stride(1) != 1 or not f.is_cuda:
                raise ValueError("frames must be 2-D uint8 CUDA tensors with unit column stride")
            dims[i] = Dims(f.shape[1], f.shape[0], f.stride(0))
            fptr[i] = f.data_ptr()
        dev = frames[0].device
        outs = [[torch.empty((num_cells(d.w, d.h, cell), 4), dtype=torch.int32, device=dev) for d in dims]
                for _ in range(npar)]
        counts = torch.empty((npar, n), dtype=torch.int32, device=dev)
        optr = (ctypes.c_void_p * (npar * n))(*[o.data_ptr() for row in outs for o in row])
        th = (ctypes.c_int * npar)(*[p[0] for p in params])
        ar = (ctypes.c_int * npar)(*[p[1] for p in params])
        self._check(self.lib.vio_detect_sweep(self.ctx, fptr, dims, n, th, ar, npar, cell, levels, optr,
                                              ctypes.c_void_p(counts.data_ptr()), _stream_handle(stream)))
        self._last_dims = [(d.w, d.h) for d in dims]
        return outs, counts

    def detect_sweep_ptrs(self, fptr, dims, n, th, ar, npar, cell, levels, optr, counts_ptr, stream_handle):
        """Pre-marshalled sweep call (ctypes arrays), for timing loops."""
        self._check(self.lib.vio_detect_sweep(self.ctx, fptr, dims, n, th, ar, npar, cell, levels, optr, counts_ptr,
                                              stream_handle))

    def detect_ptrs(self, fptr, dims, n, thresh, arc_len, cell, levels, optr, counts_ptr, stream_handle):
        """Pre-marshalled call (ctypes arrays), for timing loops."""
        self._check(self.lib.vio_detect(self.ctx, fptr, dims, n, thresh, arc_len, cell, levels, optr,
                                        counts_ptr, stream_handle))

    def detect_host(self, frames, thresh: int, arc_len: int, cell: int, levels: int,
                    outs=None, counts=None, stream=None):
        """frames: list of 2-D uint8 numpy arrays (host).  Returns numpy results."""
        n = len(frames)
        dims = (Dims * n)()
        fptr = (ctypes.c_void_p * n)()
        for i, f in enumerate(frames):
            if f.dtype != np.uint8 or f.ndim != 2 or f.strides[1] != 1:
                raise ValueError("frames must be 2-D uint8 arrays with unit column stride")
            dims[i] = Dims(f.shape[1], f.shape[0], f.strides[0])
            fptr[i] = f.ctypes.data
        if outs is None:
            outs = [np.empty((num_cells(d.w, d.h, cell), 4), dtype=np.int32) for d in dims]
        if counts is None:
            counts = np.empty(n, dtype=np.int32)
        optr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
        self._check(self.lib.vio_detect_host(self.ctx, fptr, dims, n, thresh, arc_len, cell, levels, optr,
                                             ctypes.c_void_p(counts.ctypes.data),
                                             _stream_handle(stream) if stream is not None else ctypes.c_void_p(0)))
        self._last_dims = [(d.w, d.h) for d in dims]
        return outs, counts

    def detect_host_batch(self, batch: "HostBatch", thresh: int, arc_len: int, cell: int, levels: int,
                          stream=None, pipelined: bool = False):
        """vio_detect_host (or, pipelined, vio_detect_host_async) on a
        HostBatch: no per-call marshalling."""
        fn = self.lib.vio_detect_host_async if pipelined else self.lib.vio_detect_host
        self._check(fn(self.ctx, batch.fptr, batch.dims, batch.n, thresh, arc_len, cell, levels, batch.optr,
                       batch.cptr, _stream_handle(stream) if stream is not None else ctypes.c_void_p(0)))

    def detect_host_async(self, frames, thresh: int, arc_len: int, cell: int, levels: int, outs, counts=None,
                          stream=None):
        """Asynchronous host-buffer detection: frames are 2-D uint8 numpy
        arrays (pinned or pageable), outs (and counts) numpy views of pinned
        memory that the device writes; valid after sync(stream)."""
        n = len(frames)
        dims = (Dims * n)()
        fptr = (ctypes.c_void_p * n)()
        for i, f in enumerate(frames):
            if f.dtype != np.uint8 or f.ndim != 2 or f.strides[1] != 1:
                raise ValueError("frames must be 2-D uint8 arrays with unit column stride")
            dims[i] = Dims(f.shape[1], f.shape[0], f.strides[0])
            fptr[i] = f.ctypes.data
        optr = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
        cptr = ctypes.c_void_p(counts.ctypes.data) if counts is not None else None
        self._check(self.lib.vio_detect_host_async(self.ctx, fptr, dims, n, thresh, arc_len, cell, levels, optr, cptr,
                                                   _stream_handle(stream) if stream is not None
                                                   else ctypes.c_void_p(0)))
        return outs, counts

    def stage_ms(self) -> tuple[float, float, float]:
        """(pyramid, fused detect, decode) device ms of the last call."""
        ms = (ctypes.c_float * 3)()
        self._check(self.lib.vio_stage_ms(self.ctx, ms))
        return ms[0], ms[1], ms[2]

    def copy_level(self, frame: int, level: int, stream=None) -> np.ndarray:
        """Level `level` of frame `frame` of the most recent detection call
        (host copy; waits for the stream)."""
        d = self._last_dims_of(frame)
        w, h = d[0] >> level, d[1] >> level
        out = np.empty((h, w), dtype=np.uint8)
        self._check(self.lib.vio_copy_level(self.ctx, frame, level, ctypes.c_void_p(out.ctypes.data), w,
                                            _stream_handle(stream)))
        self.sync(stream)
        return out

    def _last_dims_of(self, frame: int):
        dims = getattr(self, "_last_dims", None)
        if dims is None or not 0 <= frame < len(dims):
            raise VioError(1, "no such frame in the most recent detection")
        return dims[frame]

    def sync(self, stream=None):
        self._check(self.lib.vio_sync(self.ctx, _stream_handle(stream)))

    # ---- serving -------------------------------------------------------------
    def serve_start(self, **kw):
        """Starts the context's scheduler; keyword arguments override the
        fields of vio_serve_config (thresh, arc_len, cell_size, levels,
        max_batch, max_wait_us, lanes, mem_budget_bytes, queue_capacity,
        keep_results)."""
        cfg = ServeConfig()
        self.lib.vio_serve_config_default(ctypes.byref(cfg))
        for k, v in kw.items():
            setattr(cfg, k, v)
        self.serve_cfg = cfg
        self._check(self.lib.vio_serve_start(self.ctx, ctypes.byref(cfg)))

    def submit(self, stream_id: int, frame: np.ndarray) -> int:
        """Queues a host frame (kept alive by the caller until it completes)."""
        if frame.dtype != np.uint8 or frame.ndim != 2 or frame.strides[1] != 1:
            raise ValueError("frame must be a 2-D uint8 array with unit column stride")
        t = ctypes.c_uint64()
        d = Dims(frame.shape[1], frame.shape[0], frame.strides[0])
        s = self.lib.vio_submit(self.ctx, stream_id, ctypes.c_void_p(frame.ctypes.data), d, ctypes.byref(t))
        if s != 0:
            raise VioError(s, self.lib.vio_status_str(s).decode())
        return t.value

    def submit_raw(self, stream_id: int, ptr: int, dims: Dims) -> tuple[int, int]:
        """(status, ticket) without raising, for load generators."""
        t = ctypes.c_uint64()
        s = self.lib.vio_submit(self.ctx, stream_id, ctypes.c_void_p(ptr), dims, ctypes.byref(t))
        return s, t.value

    def poll(self, ticket: int, w: int, h: int):
        """(done, cells (ncells, 4) int32 or None, count)."""
        cfg = self.serve_cfg
        out = np.empty((num_cells(w, h, cfg.cell_size), 4), dtype=np.int32)
        cnt = ctypes.c_int32()
        done = ctypes.c_int()
        self._check(self.lib.vio_poll(self.ctx, ticket, ctypes.c_void_p(out.ctypes.data), ctypes.byref(cnt),
                                      ctypes.byref(done)))
        return (True, out, cnt.value) if done.value else (False, None, 0)

    def drain(self, timeout_ms: int = 60000):
        self._check(self.lib.vio_serve_drain(self.ctx, timeout_ms))

    def serve_stats(self) -> dict:
        st = ServeStats()
        self._check(self.lib.vio_serve_stats(self.ctx, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServeStats._fields_}

    def serve_stop(self):
        self._check(self.lib.vio_serve_stop(self.ctx))

    def set_variant(self, variant: int | None, cta_per_sm: int = 0):
        """Pins a tile variant (and a CTA count per SM, 0 = as many as fit);
        None unpins both."""
        if variant is None:
            self._check(self.lib.vio_set_tuning(self.ctx, None))
            return
        t = Tuning(0, 0, cta_per_sm, variant, 0, 0)
        self._check(self.lib.vio_set_tuning(self.ctx, ctypes.byref(t)))

    def tuning_full(self) -> dict:
        """The launch configuration of the most recent detection."""
        t = Tuning()
        self._check(self.lib.vio_get_tuning(self.ctx, ctypes.byref(t)))
        return {name: getattr(t, name) for name, _ in Tuning._fields_}

    def autotune_log(self) -> list[dict]:
        """What the most recent tuning run timed: configuration and ms per call."""
        n = self.lib.vio_autotune_log(self.ctx, None, None, 0)
        cfgs = (Tuning * max(1, n))()
        ms = (ctypes.c_float * max(1, n))()
        self.lib.vio_autotune_log(self.ctx, cfgs, ms, n)
        return [{**{name: getattr(cfgs[i], name) for name, _ in Tuning._fields_}, "ms": round(ms[i], 5)}
                for i in range(n)]

    def config(self) -> Config:
        c = Config()
        self._check(self.lib.vio_get_config(self.ctx, ctypes.byref(c)))
        return c

    def tuning(self) -> tuple[int, int, int]:
        t = Tuning()
        self._check(self.lib.vio_get_tuning(self.ctx, ctypes.byref(t)))
        return t.tile_w, t.tile_h, t.variant
