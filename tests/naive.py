"""A second, deliberately different formulation of the detector, in pure Python.

Used only to pin the C oracle on tiny images.  It is written from the same
passages of the paper (Section II-B..II-D, Eq. 1, Algorithm 1) but takes
other routes wherever one exists:

* the circle is derived from the midpoint-circle construction of radius 3
  and sorted by angle, instead of being typed in as a table;
* the segment test rotates the label list and looks for a run as a substring;
* SAD-A is the maximum over *all* homogeneous arcs of length >= N (the sum of
  non-negative terms is largest on the maximal run);
* MT is a brute-force scan of every threshold;
* NMS compares each pixel against an explicit neighbour list;
* NMS-C sorts all candidates per cell by (-score, level, y, x).
"""
from __future__ import annotations

import math

import numpy as np


def bresenham_circle_r3() -> list[tuple[int, int]]:
    """Midpoint circle of radius 3 (16 points), clockwise from the top in image
    coordinates (y grows downwards)."""
    pts = set()
    x, y, d = 0, 3, 1 - 3
    while x <= y:
        for (a, b) in ((x, y), (y, x), (-x, y), (-y, x), (x, -y), (y, -x), (-x, -y), (-y, -x)):
            pts.add((a, b))
        x += 1
        if d < 0:
            d += 2 * x + 1
        else:
            y -= 1
            d += 2 * (x - y) + 1
    # clockwise on screen from (0,-3): angle measured from "up" towards "right"
    return sorted(pts, key=lambda p: math.atan2(p[0], -p[1]) % (2 * math.pi))


CIRCLE = bresenham_circle_r3()


def labels(img, x, y, t):
    c = int(img[y][x])
    out = []
    for dx, dy in CIRCLE:
        v = int(img[y + dy][x + dx])
        out.append("b" if v > c + t else ("d" if v < c - t else "s"))
    return out


def has_run(lab, pol, n):
    s = "".join(lab)
    return pol * n in s + s


def is_corner(img, x, y, t, n):
    lab = labels(img, x, y, t)
    return has_run(lab, "b", n) or has_run(lab, "d", n)


def score(img, x, y, t, n, mode):
    h, w = len(img), len(img[0])
    if not (3 <= x < w - 3 and 3 <= y < h - 3):
        return 0
    if not is_corner(img, x, y, t, n):
        return 0
    c = int(img[y][x])
    diffs = [abs(int(img[y + dy][x + dx]) - c) for dx, dy in CIRCLE]
    if mode == 0:
        return sum(diffs)
    if mode == 1:
        lab = labels(img, x, y, t)
        best = 0
        for pol in "bd":
            for s in range(16):
                for ln in range(n, 17):
                    idx = [(s + j) % 16 for j in range(ln)]
                    if all(lab[i] == pol for i in idx):
                        best = max(best, sum(diffs[i] for i in idx))
        return best
    best = 0
    for tt in range(0, 256):
        if tt >= t and is_corner(img, x, y, tt, n):
            best = tt
    return best


def pyramid(img, levels):
    out = [np.asarray(img, dtype=np.int64)]
    for _ in range(1, levels):
        a = out[-1]
        h, w = a.shape[0] // 2 * 2, a.shape[1] // 2 * 2
        b = a[:h, :w]
        s = b[0::2, 0::2] + b[0::2, 1::2] + b[1::2, 0::2] + b[1::2, 1::2]
        out.append((s + 2) // 4)
    return [o.astype(np.uint8) for o in out]


def neighbours(radius):
    return [(dx, dy) for dy in range(-radius, radius + 1) for dx in range(-radius, radius + 1)
            if (dx, dy) != (0, 0)]


NEIGHBOURS = neighbours(1)


def nms(s, radius=1):
    h, w = len(s), len(s[0])
    out = [[0] * w for _ in range(h)]
    nbs = neighbours(radius)
    for y in range(h):
        for x in range(w):
            v = s[y][x]
            if v <= 0:
                continue
            nb = [s[y + dy][x + dx] if 0 <= x + dx < w and 0 <= y + dy < h else 0 for dx, dy in nbs]
            if all(v >= q for q in nb):
                out[y][x] = v
    return out


def nms3(s):
    return nms(s, 1)


def detect(img, t, n, cell, levels, mode=0, radius=1):
    img = np.asarray(img, dtype=np.uint8)
    h, w = img.shape
    gw, gh = -(-w // cell), -(-h // cell)
    cands = {}
    for k, lev in enumerate(pyramid(img, levels)):
        L = lev.tolist()
        hk, wk = len(L), len(L[0]) if L else 0
        sm = [[score(L, x, y, t, n, mode) for x in range(wk)] for y in range(hk)]
        m = nms(sm, radius) if hk and wk else []
        for y in range(hk):
            for x in range(wk):
                if m[y][x] > 0:
                    cid = ((y << k) // cell) * gw + ((x << k) // cell)
                    cands.setdefault(cid, []).append((-m[y][x], k, y, x))
    out = np.tile(np.array([-1, -1, -1, 0], dtype=np.int32), (gw * gh, 1))
    for cid, lst in cands.items():
        ns, k, y, x = sorted(lst)[0]
        out[cid] = (x << k, y << k, k, -ns)
    return out
