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
