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
