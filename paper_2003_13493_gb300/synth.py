"""Seeded synthetic grayscale frames (the input recipe for every test and benchmark).

This module draws pixels and nothing else: it holds none of the detector's
arithmetic, so both the CPU oracle and the CUDA path can be fed from it.

The frames stand in for the EuRoC Machine Hall sequences the paper evaluates on
(Section III): 8-bit grayscale, smooth texture with sharp-edged objects.

Recipe (integer-only, so the bytes are identical on every host):

* Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014), used counter-style: draw ``i``
  of a frame with seed ``s`` is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``.
* Texture: value noise on an 8-pixel lattice.  Each lattice value is
  ``128 + round(30 * (sum of 12 uniforms - 6))`` (Irwin-Hall approximation of a
  normal with mean 128, std 30), uniforms taken as the top 16 bits of a draw,
  rounding half up in 1/65536 fixed point.  Pixels are bilinear with integer
  weights ``(x mod 8)/8``, rounded half up.
* Shapes: ``n_shapes`` objects painted in order, each a rectangle or a triangle
  with probability 1/2, side/extent uniform in ``[8, max(8, min(W, H) // 4)]``,
  fill uniform in ``0..255``.  Triangles are rasterised with integer edge
  functions at pixel centres, edges inclusive.
* Finally every value is clamped to ``0..255``.
"""
from __future__ import annotations

import hashlib

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

#: Frame sizes of the mixed-size batch (width, height).
MIXED_SIZES = ((640, 480), (752, 480), (1280, 720), (1920, 1080))


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream for ``seed``."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _lattice(w: int, h: int, seed: int) -> tuple[np.ndarray, int]:
    lw, lh = (w + 7) // 8 + 1, (h + 7) // 8 + 1
    n = 12 * lw * lh
    d = splitmix64(seed, n).reshape(lh, lw, 12)
    u = (d >> np.uint64(48)).astype(np.int64)
    s = u.sum(axis=2) - 6 * 65536
    # round half up of 30*s/65536 (floor division keeps it exact for negatives)
    val = 128 + ((30 * s + 32768) >> 16)
    return val, n


def _texture(w: int, h: int, lat: np.ndarray) -> np.ndarray:
    xs = np.arange(w)
    ys = np.arange(h)
    gx, fx = xs >> 3, xs & 7
    gy, fy = ys >> 3, ys & 7
    l00 = lat[gy][:, gx]
    l01 = lat[gy][:, gx + 1]
    l10 = lat[gy + 1][:, gx]
    l11 = lat[gy + 1][:, gx + 1]
    top = l00 * (8 - fx)[None, :] + l01 * fx[None, :]
    bot = l10 * (8 - fx)[None, :] + l11 * fx[None, :]
    return (top * (8 - fy)[:, None] + bot * fy[:, None] + 32) >> 6


def _u(d: np.uint64, m: int) -> int:
    """Uniform integer in ``0..m-1`` from the top 32 bits of a draw."""
    return int(d >> np.uint64(32)) % m


def _paint_shapes(img: np.ndarray, seed: int, n_shapes: int, start: int) -> None:
    h, w = img.shape
    smax = max(8, min(w, h) // 4)
    span = smax - 8 + 1
    d = splitmix64(seed, 8 * n_shapes, start).reshape(n_shapes, 8)
    for k in range(n_shapes):
        dk = d[k]
        fill = int(dk[7] & np.uint64(255))
        if int(dk[0] >> np.uint64(63)) == 0:  # rectangle
            x0, y0 = _u(dk[1], w), _u(dk[2], h)
            sw, sh = 8 + _u(dk[3], span), 8 + _u(dk[4], span)
            img[y0:min(h, y0 + sh), x0:min(w, x0 + sw)] = fill
            continue
        cx, cy = _u(dk[1], w), _u(dk[2], h)
        e = 8 + _u(dk[3], span)
        offs = []
        for j in (4, 5, 6):
            lo = int(dk[j] & np.uint64(0xFFFFFFFF))
            hi = int(dk[j] >> np.uint64(32))
            offs.append((cx + lo % (2 * e + 1) - e, cy + hi % (2 * e + 1) - e))
        (ax, ay), (bx, by), (qx, qy) = offs
        area = (bx - ax) * (qy - ay) - (by - ay) * (qx - ax)
        if area == 0:
            continue
        xlo, xhi = max(0, min(ax, bx, qx)), min(w - 1, max(ax, bx, qx))
        ylo, yhi = max(0, min(ay, by, qy)), min(h - 1, max(ay, by, qy))
        if xlo > xhi or ylo > yhi:
            continue
        # pixel centres (2x+1, 2y+1) against doubled vertices
        px = (2 * np.arange(xlo, xhi + 1) + 1)[None, :]
        py = (2 * np.arange(ylo, yhi + 1) + 1)[:, None]
        inside = np.ones((yhi - ylo + 1, xhi - xlo + 1), dtype=bool)
        sgn = 1 if area > 0 else -1
        for (x1, y1), (x2, y2) in (((ax, ay), (bx, by)), ((bx, by), (qx, qy)),
                                   ((qx, qy), (ax, ay))):
            ef = (2 * x2 - 2 * x1) * (py - 2 * y1) - (2 * y2 - 2 * y1) * (px - 2 * x1)
            inside &= sgn * ef >= 0
        img[ylo:yhi + 1, xlo:xhi + 1][inside] = fill


def make_frame(w: int, h: int, seed: int, n_shapes: int = 40) -> np.ndarray:
    """One ``h x w`` uint8 frame (C-contiguous, row pitch ``w``)."""
    if w < 1 or h < 1:
        raise ValueError("frame size must be positive")
    lat, used = _lattice(w, h, seed)
    img = _texture(w, h, lat)
    _paint_shapes(img, seed, n_shapes, used)
    return np.ascontiguousarray(np.clip(img, 0, 255).astype(np.uint8))


def frame_sha256(img: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest()


def mixed_batch(first_seed: int = 2, per_size: int = 16, n_shapes: int = 40):
    """The mixed-size batch: ``per_size`` frames of each size in ``MIXED_SIZES``,
    seeds ``first_seed, first_seed+1, ...`` in size-major order."""
    frames = []
    seed = first_seed
    for (w, h) in MIXED_SIZES:
        for _ in range(per_size):
            frames.append(make_frame(w, h, seed, n_shapes))
            seed += 1
    return frames


# ---- frame pairs for the feature tracker ------------------------------------
#
# A pair is a previous frame and a next frame that shows the same scene moved
# by (dx, dy) pixels and with its intensities mapped by v -> gain * v + offset.
# The scene is a sum of seeded plane waves (smooth, textured everywhere, no
# flat areas), evaluated in float64 and rounded to 8 bits, so that sub-pixel
# motion has an exact ground truth.  Unlike make_frame the bytes may differ in
# the last bit between hosts (libm), which does not matter: the tracker and
# its oracle always read the bytes generated on the same host.

def _waves(seed: int, n: int = 6):
    d = splitmix64(seed ^ 0x5A5A5A5A, 4 * n)
    u = (d >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    freq = 0.05 + 0.25 * u[0::4]
    ang = 2.0 * np.pi * u[1::4]
    phase = 2.0 * np.pi * u[2::4]
    amp = 12.0 + 16.0 * u[3::4]
    return freq * np.cos(ang), freq * np.sin(ang), phase, amp


def smooth_frame(w: int, h: int, seed: int, dx: float = 0.0, dy: float = 0.0, gain: float = 1.0,
                 offset: float = 0.0) -> np.ndarray:
    """The scene of `seed` moved by (dx, dy): pixel (x, y) shows scene point
    (x - dx, y - dy); intensities gain * v + offset, rounded and clamped."""
    kx, ky, phase, amp = _waves(seed)
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    x -= dx
    y -= dy
    v = np.full((h, w), 128.0)
    for i in range(len(kx)):
        v += amp[i] * np.sin(kx[i] * x + ky[i] * y + phase[i]) * (0.8 if i % 2 else 1.0)
    v = gain * v + offset
    return np.ascontiguousarray(np.clip(np.floor(v + 0.5), 0, 255).astype(np.uint8))


def shift_frame(img: np.ndarray, dx: int, dy: int, fill: int = 0) -> np.ndarray:
    """img moved by whole pixels: out[y, x] = img[y - dy, x - dx]."""
    h, w = img.shape
    out = np.full_like(img, fill)
    ys, yd = (slice(0, h - dy), slice(dy, h)) if dy >= 0 else (slice(-dy, h), slice(0, h + dy))
    xs, xd = (slice(0, w - dx), slice(dx, w)) if dx >= 0 else (slice(-dx, w), slice(0, w + dx))
    out[yd, xd] = img[ys, xs]
    return out
