"""Plain fp64 oracle of the feature tracker (Section II-E, Eqs. 2-6).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module; the library never imports it.
It shares no code with the CUDA path.

The tracker is the approximated simultaneous inverse compositional
Lucas-Kanade algorithm: a translation t = (t_x, t_y) (Eq. 2) and an affine
intensity change (alpha, beta), so that the next image I matches the
template T as  I(x + t) ~ (1 + alpha) T(x) + beta  over a square patch N
around the feature.  Per pyramid level, coarse to fine:

  * the template patch and its gradients are sampled once (bilinear
    interpolation of the previous image; gradients by central differences
    of the interpolated template grid);
  * U(x) = [(1+alpha) dT/dx, (1+alpha) dT/dy, T(x), 1]   (Eq. 4) and
    H = sum_x U U^T (Eq. 6) are formed once per level with the appearance
    estimate at the start of the level (the "approximated" variant: the
    Hessian is not rebuilt when alpha changes);
  * every iteration samples I at x + t, forms the residual
    r = I(x + t) - (1+alpha) T(x) - beta, solves
    dq = H^-1 sum_x U r (Eq. 6) and updates  t <- t - dt  (inverse
    composition of the translation), alpha <- alpha + d_alpha,
    beta <- beta + d_beta; the level ends after max_iters iterations or when
    |dt| < min_update;
  * the translation doubles from one level to the next finer one.

Readings where the paper is silent (the same on both sides):
  * a level-0 position x maps to level k at (x + 0.5) / 2^k - 0.5 (pixel
    centres of the 2x2-mean pyramid);
  * the patch is P x P samples at offsets i - (P - 1) / 2, P = patch_fine on
    level 0 and patch_coarse on the coarser levels (the paper uses 16 x 16 on
    high and 8 x 8 on low resolutions);
  * bilinear samples need 0 <= x <= W_k - 2 and 0 <= y <= H_k - 2; a sample
    outside, or a Hessian that is not positive definite, loses the track;
  * parameters the model does not estimate stay 0 (Table VI's subsets);
  * the reported residual is the root mean square of r in the last
    iteration on level 0; a lost track reports its estimate so far, scaled to
    level-0 pixels.
"""
from __future__ import annotations

import numpy as np

GAIN, OFFSET = 1, 2  # model bits: estimate alpha, estimate beta

TRACKED, LOST = 1, 0


def pyramid(img: np.ndarray, levels: int) -> list[np.ndarray]:
    """The detector's pyramid (Section II-B), from the C oracle."""
    from . import pyramid as _pyramid

    return _pyramid(np.ascontiguousarray(img, dtype=np.uint8), levels)


def inside(img: np.ndarray, x: np.ndarray, y: np.ndarray) -> bool:
    h, w = img.shape
    return bool(np.all((x >= 0) & (x <= w - 2) & (y >= 0) & (y <= h - 2)))


def bilinear(img: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Bilinear interpolation at (x, y); the caller checked `inside`."""
    a = np.asarray(img, dtype=np.float64)
    x0 = np.floor(x).astype(np.int64)
    y0 = np.floor(y).astype(np.int64)
    fx = x - x0
    fy = y - y0
    return ((1 - fx) * (1 - fy) * a[y0, x0] + fx * (1 - fy) * a[y0, x0 + 1]
            + (1 - fx) * fy * a[y0 + 1, x0] + fx * fy * a[y0 + 1, x0 + 1])


def active(model: int) -> list[int]:
    """Indices into q = [t_x, t_y, alpha, beta] that the model estimates."""
    return [0, 1] + ([2] if model & GAIN else []) + ([3] if model & OFFSET else [])


def track_one(prev_pyr, next_pyr, x: float, y: float, *, patch_fine: int = 16, patch_coarse: int = 8,
              max_iters: int = 30, min_update: float = 0.01, model: int = GAIN | OFFSET):
    """Tracks one feature at level-0 position (x, y) of the previous frame.

    Returns (x', y', alpha, beta, status, iterations, residual)."""
    levels = len(prev_pyr)
    t = np.zeros(2)
    alpha = beta = 0.0
    iters = 0
    residual = 0.0
    idx = active(model)

    def lost(k):  # the estimate so far, in level-0 pixels
        return x + t[0] * 2 ** k, y + t[1] * 2 ** k, alpha, beta, LOST, iters, residual

    for k in range(levels - 1, -1, -1):
        P = patch_fine if k == 0 else patch_coarse
        T_img, I_img = prev_pyr[k], next_pyr[k]
        cx = (x + 0.5) / 2 ** k - 0.5
        cy = (y + 0.5) / 2 ** k - 0.5
        off = np.arange(-1, P + 1) - (P - 1) / 2.0          # template grid with a 1-sample border
        gx, gy = np.meshgrid(cx + off, cy + off)             # gx[j, i]: row j, column i
        if not inside(T_img, gx, gy):
            return lost(k)
        Tg = bilinear(T_img, gx, gy)
        T = Tg[1:-1, 1:-1]
        Tx = (Tg[1:-1, 2:] - Tg[1:-1, :-2]) / 2.0
        Ty = (Tg[2:, 1:-1] - Tg[:-2, 1:-1]) / 2.0
        px, py = gx[1:-1, 1:-1], gy[1:-1, 1:-1]
        # Eq. 4 with the appearance estimate at the start of the level
        U = np.stack([(1 + alpha) * Tx, (1 + alpha) * Ty, T, np.ones_like(T)], axis=-1).reshape(-1, 4)
        Ua = U[:, idx]
        H = Ua.T @ Ua                                         # Eq. 6
        try:
            np.linalg.cholesky(H)
        except np.linalg.LinAlgError:
            return lost(k)
        for _ in range(max_iters):
            qx, qy = px + t[0], py + t[1]
            if not inside(I_img, qx, qy):
                return lost(k)
            r = (bilinear(I_img, qx, qy) - (1 + alpha) * T - beta).reshape(-1)
            residual = float(np.sqrt(np.mean(r * r)))
            dq = np.linalg.solve(H, Ua.T @ r)                 # Eq. 6
            full = np.zeros(4)
            full[idx] = dq
            t = t - full[:2]
            alpha += full[2]
            beta += full[3]
            iters += 1
            if np.hypot(full[0], full[1]) < min_update:
                break
        if k > 0:
            t = 2.0 * t
    return x + t[0], y + t[1], alpha, beta, TRACKED, iters, residual


def track(prev: np.ndarray, nxt: np.ndarray, pts: np.ndarray, *, levels: int = 3, **kw) -> np.ndarray:
    """Tracks every row (x, y) of pts; returns rows
    (x', y', alpha, beta, status, iterations, residual) as float64."""
    pp, nn = pyramid(prev, levels), pyramid(nxt, levels)
    out = np.zeros((len(pts), 7))
    for i, (x, y) in enumerate(np.asarray(pts, dtype=np.float64)):
        out[i] = track_one(pp, nn, float(x), float(y), **kw)
    return out
