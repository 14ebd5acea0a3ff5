"""CPU models of the bit tricks the fused kernel relies on, checked
exhaustively over their input ranges (no GPU, no oracle involved)."""
import numpy as np

M7 = 0x7F7F7F7F


def byte_gt(d: int, t: int) -> int:
    """The kernel's carry-free byte-wise compare d > t (flag in bit 7)."""
    high = t >= 128
    k7 = ((255 if high else 127) - t) * 0x01010101
    f = ((d & M7) + k7) & 0xFFFFFFFF
    f = (f & d) if high else (f | d)
    return f & 0x80808080


def test_byte_compare_exact():
    for t in range(256):
        for d0 in range(256):
            ds = [d0, (d0 * 7 + 3) & 255, (d0 * 13 + 5) & 255, 255 - d0]
            f = byte_gt(sum(v << (8 * i) for i, v in enumerate(ds)), t)
            for i, v in enumerate(ds):
                assert bool((f >> (8 * i + 7)) & 1) == (v > t), (t, v)


def test_imad_labels_exact():
    """One multiply-add gives both Eq. 1 labels: bit 15 = brighter, bit 31 = darker."""
    v = np.arange(256, dtype=np.uint64)
    for t in range(256):
        for c in range(256):
            k = ((0x7FFF - c - t) & 0xFFFF) | (((0x7FFF + c - t) & 0xFFFF) << 16)
            w = (np.uint64(k) + v * np.uint64(0xFFFF0001)) & np.uint64(0xFFFFFFFF)
            assert np.array_equal((w >> np.uint64(15)) & np.uint64(1) == 1, np.arange(256) > c + t)
            assert np.array_equal((w >> np.uint64(31)) & np.uint64(1) == 1, np.arange(256) < c - t)


def _has_run(m, n):
    s = format(m, "016b")[::-1]
    return "1" * n in s + s


def test_coarse_test_never_drops_a_corner():
    """Every 16-point mask with a cyclic run of n (9..16) passes the compass
    test the kernel uses: two adjacent compass points for n <= 11, three of
    four for n >= 12."""
    for n in range(9, 17):
        for m in range(1 << 16):
            if not _has_run(m, n):
                continue
            f = [(m >> p) & 1 for p in (0, 4, 8, 12)]
            keep = sum(f) >= 3 if n >= 12 else (f[0] | f[2]) & (f[1] | f[3])
            assert keep, (hex(m), n)


def _byte_perm(a, b, sel):
    """__byte_perm(a, b, sel): result byte i is byte (sel >> 4i) & 7 of b:a."""
    src = a | (b << 32)
    return sum(((src >> (8 * ((sel >> (4 * i)) & 7))) & 0xFF) << (8 * i) for i in range(4))


def test_coarse_shifts_select_the_circle_columns():
    """The byte selections of coarse4/coarse8: with C = pixels x..x+3 and
    its neighbour words L, R, 0x6543 gives x+3.., 0x4321 gives x-3.., 0x5432
    gives x+2.. from (C, R) and x-2.. from (L, C)."""
    row = list(range(12))  # pixel values = their column; C holds columns 4..7
    word = lambda i: sum(row[i + j] << (8 * j) for j in range(4))
    L, C, R = word(0), word(4), word(8)
    cols = lambda w: [(w >> (8 * j)) & 0xFF for j in range(4)]
    assert cols(_byte_perm(C, R, 0x6543)) == [7, 8, 9, 10]
    assert cols(_byte_perm(L, C, 0x4321)) == [1, 2, 3, 4]
    assert cols(_byte_perm(C, R, 0x5432)) == [6, 7, 8, 9]
    assert cols(_byte_perm(L, C, 0x5432)) == [2, 3, 4, 5]


def _eight(f):
    """coarse8's keep formula on the flags of N, NE, E, SE, S, SW, W, NW."""
    fn, fne, fe, fse, fs, fsw, fw, fnw = f
    xne, xse, xsw, xnw = fn & fne & fe, fe & fse & fs, fs & fsw & fw, fw & fnw & fn
    return ((xne | xsw) & (fse | fnw)) | ((xse | xnw) & (fne | fsw))


def test_eight_point_formula_is_four_consecutive():
    """The grouped formula equals 'four cyclically consecutive of the eight'
    for all 256 flag patterns, and implies the compass two-adjacent rule."""
    for m in range(256):
        f = [(m >> i) & 1 for i in range(8)]
        runs = any(all(f[(s + j) % 8] for j in range(4)) for s in range(8))
        assert bool(_eight(f)) == runs, m
        if runs:
            assert (f[0] | f[4]) & (f[2] | f[6])


def test_eight_point_test_never_drops_a_corner():
    """Every 16-point mask with a cyclic run of n (9..16) has four
    consecutive even points (0, 2, .., 14) set, so coarse8 keeps it."""
    for n in range(9, 17):
        for m in range(1 << 16):
            if _has_run(m, n):
                assert _eight([(m >> (2 * i)) & 1 for i in range(8)]), (hex(m), n)


def test_even_circle_points_are_compass_and_diagonals():
    """The Bresenham circle of radius 3 (points numbered clockwise from the
    top, as in FAST) has its even points at the compass points and the four
    (+-2, +-2) diagonals, in the cyclic order coarse8 assumes."""
    circle = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
              (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3)]
    ring = {(x, y) for x in range(-3, 4) for y in range(-3, 4) if 2.5 <= (x * x + y * y) ** 0.5 < 3.5}
    assert set(circle) == ring and len(circle) == 16
    # clockwise from the top in image coordinates (y down)
    ang = [np.arctan2(x, -y) % (2 * np.pi) for x, y in circle]
    assert ang == sorted(ang)
    assert circle[0::2] == [(0, -3), (2, -2), (3, 0), (2, 2), (0, 3), (-2, 2), (-3, 0), (-2, -2)]


def test_arc_starts_doubling():
    """arc_starts: runs of n from three AND-shift doublings plus an overlap."""
    for n in range(9, 17):
        for m in range(0, 1 << 16, 7):
            r = (m * 0x10001) & 0xFFFFFFFF
            r &= r >> 1
            r &= r >> 2
            r &= r >> 4
            r &= r >> (n - 8)
            assert bool(r & 0xFFFF) == _has_run(m, n)


# ---- MT score by packed window minima ----------------------------------------

def _lanes(w):
    return w & 0xFFFF, w >> 16


def _pack(lo, hi):
    return (lo & 0xFFFF) | ((hi & 0xFFFF) << 16)


def _min16(a, b):
    return _pack(min(_lanes(a)[0], _lanes(b)[0]), min(_lanes(a)[1], _lanes(b)[1]))


def _perm5432(a, b):  # __byte_perm(a, b, 0x5432): high half of a, low half of b
    return (a >> 16) | ((b & 0xFFFF) << 16)


def mt_packed(v, c, bright, n):
    """The kernel's MT: biased 16-bit differences two per word, window minima
    by doubling, the largest over all 16 starts, minus the bias and 1."""
    c2 = c * 0x00010001
    D = []
    for j in range(8):
        V = v[2 * j] | (v[2 * j + 1] << 16)
        D.append(((V + (0x01000100 - c2)) if bright else ((0x01000100 + c2) - V)) & 0xFFFFFFFF)
    M2 = [_min16(D[j], _perm5432(D[j], D[(j + 1) & 7])) for j in range(8)]
    M4 = [_min16(M2[j], M2[(j + 1) & 7]) for j in range(8)]
    M8 = [_min16(M4[j], M4[(j + 2) & 7]) for j in range(8)]
    r = n - 8
    W = []
    for j in range(8):
        S = _perm5432(M8[(j + r // 2) & 7], M8[(j + r // 2 + 1) & 7]) if r & 1 else M8[(j + r // 2) & 7]
        W.append(_min16(M8[j], S))
    best = max(max(_lanes(w)) for w in W)
    return best - 257


def _mt_brute(v, c, t, n):
    best = 0
    for tt in range(t, 256):
        b = sum(1 << i for i in range(16) if v[i] > c + tt)
        d = sum(1 << i for i in range(16) if v[i] < c - tt)
        if _has_run(b, n) or _has_run(d, n):
            best = tt
    return best


def test_mt_packed_window_minima_match_brute_force():
    rng = np.random.default_rng(5)
    checked = 0
    while checked < 3000:
        n = int(rng.integers(9, 17))
        t = int(rng.integers(0, 60))
        c = int(rng.integers(0, 256))
        bright = bool(rng.integers(0, 2))
        # an arc of n points beyond the threshold at a random start, the rest random
        v = [int(x) for x in rng.integers(0, 256, 16)]
        s0 = int(rng.integers(0, 16))
        for j in range(n):
            lo, hi = (c + t + 1, 255) if bright else (0, c - t - 1)
            if lo > hi:
                break
            v[(s0 + j) & 15] = int(rng.integers(lo, hi + 1))
        else:
            b = sum(1 << i for i in range(16) if v[i] > c + t)
            d = sum(1 << i for i in range(16) if v[i] < c - t)
            pol = _has_run(b, n)
            if not (pol or _has_run(d, n)):
                continue
            assert mt_packed(v, c, pol, n) == _mt_brute(v, c, t, n), (v, c, t, n)
            checked += 1


def test_mt_packed_extremes():
    # all 16 points at the far end of the range on either side
    for c in (0, 1, 128, 254, 255):
        for n in range(9, 17):
            if c < 255:
                v = [255] * 16
                assert mt_packed(v, c, True, n) == 255 - c - 1 == _mt_brute(v, c, 0, n)
            if c > 0:
                v = [0] * 16
                assert mt_packed(v, c, False, n) == c - 1 == _mt_brute(v, c, 0, n)


def test_nibble_to_byte_mask_exact():
    """SAD-A's run mask: nibble q of the 16-bit run -> 0xFF in byte i for bit i."""
    for nib in range(16):
        m = ((nib * 0x00204081) & 0x01010101) * 0xFF
        assert m == sum(0xFF << (8 * i) for i in range(4) if (nib >> i) & 1)
