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
    """The byte selections of the coarse test: with C = pixels x..x+3 and
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
    """The 8-point keep formula on the flags of N, NE, E, SE, S, SW, W, NW."""
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
    consecutive even points (0, 2, .., 14) set, so the 8-point rule keeps it."""
    for n in range(9, 17):
        for m in range(1 << 16):
            if _has_run(m, n):
                assert _eight([(m >> (2 * i)) & 1 for i in range(8)]), (hex(m), n)


def test_even_circle_points_are_compass_and_diagonals():
    """The Bresenham circle of radius 3 (points numbered clockwise from the
    top, as in FAST) has its even points at the compass points and the four
    (+-2, +-2) diagonals, in the cyclic order the 8-point rule assumes."""
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


# ---- MT score by window minima of both polarities ------------------------------

def _lanes(w):
    return w & 0xFFFF, w >> 16


def _min16(*ws):
    return min(_lanes(w)[0] for w in ws) | (min(_lanes(w)[1] for w in ws) << 16)


def best_window_min(v, c, n):
    """The kernel's window_minima8_of + best_window_min_for_arc: D_i =
    (v_i - c + 256) | (c - v_i + 256) << 16, minima of three, then of eight
    (i, i+3, i+5), a window of n = 8 + R as two windows of 8 R apart, the
    largest over the 16 windows and both lanes."""
    D = [(x - c + 256) | ((c - x + 256) << 16) for x in v]
    W3 = [_min16(D[i], D[(i + 1) % 16], D[(i + 2) % 16]) for i in range(16)]
    W8 = [_min16(W3[i], W3[(i + 3) % 16], W3[(i + 5) % 16]) for i in range(16)]
    Wn = [_min16(W8[i], W8[(i + n - 8) % 16]) for i in range(16)]
    return max(max(_lanes(w)) for w in Wn)


def mt_windows(v, c, n):
    """The MT score of a corner: largest window minimum minus the bias and 1."""
    return best_window_min(v, c, n) - 257


def _mt_brute(v, c, t, n):
    best = 0
    for tt in range(t, 256):
        b = sum(1 << i for i in range(16) if v[i] > c + tt)
        d = sum(1 << i for i in range(16) if v[i] < c - tt)
        if _has_run(b, n) or _has_run(d, n):
            best = tt
    return best


def test_mt_window_minima_match_brute_force():
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
            if not (_has_run(b, n) or _has_run(d, n)):
                continue
            assert mt_windows(v, c, n) == _mt_brute(v, c, t, n), (v, c, t, n)
            checked += 1


def test_mt_window_minima_extremes():
    # all 16 points at the far end of the range on either side
    for c in (0, 1, 128, 254, 255):
        for n in range(9, 17):
            if c < 255:
                v = [255] * 16
                assert mt_windows(v, c, n) == 255 - c - 1 == _mt_brute(v, c, 0, n)
            if c > 0:
                v = [0] * 16
                assert mt_windows(v, c, n) == c - 1 == _mt_brute(v, c, 0, n)


def test_nibble_to_byte_mask_exact():
    """SAD-A's run mask: nibble q of the 16-bit run -> 0xFF in byte i for bit i."""
    for nib in range(16):
        m = ((nib * 0x00204081) & 0x01010101) * 0xFF
        assert m == sum(0xFF << (8 * i) for i in range(4) if (nib >> i) & 1)


# ---- coarse test with shared comparisons, one warp modelled lane by lane -----

def _vabsdiff4(a, b):
    return sum(abs(((a >> (8 * i)) & 0xFF) - ((b >> (8 * i)) & 0xFF)) << (8 * i) for i in range(4))


def _gt_flags(a, b, t):
    """gt_flags: bit 7 of byte i set iff |a_i - b_i| > t (other bits left over)."""
    high = t >= 128
    k7 = ((255 if high else 127) - t) * 0x01010101
    d = _vabsdiff4(a, b)
    f = ((d & M7) + k7) & 0xFFFFFFFF
    return (f & d) if high else (f | d)


def _shfl_up(vals):
    """__shfl_up_sync(.., 1): lane l gets lane l-1's value, lane 0 keeps its own."""
    return [vals[0]] + vals[:-1]


def _shfl_down(vals):
    return vals[1:] + [vals[-1]]


def _coarse_warp(box, xw, t, rows, three, eight, radius):
    """The kernel's coarse_and_compact flags for one warp: rows score rows
    starting at r0 = 0 (box rows 3 ..), 32 lanes of 4 pixels each; returns
    kept[(row, column)] before the column and row masks."""
    word = lambda row, w: sum(int(box[row, 4 * w + j]) << (8 * j) for j in range(4))
    C = [[word(j, xw + l) for l in range(32)] for j in range(rows + 6)]
    Rw = [[word(j, xw + l + 1) for l in range(32)] for j in range(rows + 6)]
    Lw = [[word(j, xw + l - 1) for l in range(32)] for j in range(rows + 6)]
    Dv = [[_gt_flags(C[j][l], C[j + 3][l], t) for l in range(32)] for j in range(rows + 3)]
    D1, D2 = {}, {}
    for j in range(1, rows + 3):
        left = _shfl_up(C[j + 2])
        D1[j] = [_gt_flags(C[j][l], _byte_perm(C[j + 2][l], Rw[j + 2][l], 0x5432), t) for l in range(32)]
        D2[j] = [_gt_flags(C[j][l], _byte_perm(left[l], C[j + 2][l], 0x5432), t) for l in range(32)]
    kept = {}
    for i in range(rows):
        j = i + 3
        fe = [_gt_flags(C[j][l], _byte_perm(C[j][l], Rw[j][l], 0x6543), t) for l in range(32)]
        if radius == 1:
            el = _shfl_up(fe)
        else:
            el = [_gt_flags(Lw[j][l], _byte_perm(Lw[j][l], C[j][l], 0x6543), t) for l in range(32)]
        nwl = _shfl_up(D1[j - 2]) if eight else None
        ner = _shfl_down(D2[j - 2]) if eight else None
        for l in range(32):
            fw = _byte_perm(el[l], fe[l], 0x4321)
            fn, fs = Dv[i][l], Dv[j][l]
            if eight:
                fse, fsw = D1[j][l], D2[j][l]
                fnw = _byte_perm(nwl[l], D1[j - 2][l], 0x5432)
                fne = _byte_perm(D2[j - 2][l], ner[l], 0x5432)
                keep = _eight([fn, fne, fe[l], fse, fs, fsw, fw, fnw])
            elif three:
                keep = (fn & fe[l] & (fs | fw)) | (fs & fw & (fn | fe[l]))
            else:
                keep = (fn | fs) & (fe[l] | fw)
            for b in range(4):
                kept[(i, 4 * l + b)] = bool((keep >> (8 * b + 7)) & 1)
    return kept


def _coarse_reference(box, xoff, t, rows, three, eight):
    out = {}
    for i in range(rows):
        y = i + 3
        for col in range(128):
            x = col + xoff
            c = int(box[y, x])
            d = lambda dx, dy: abs(int(box[y + dy, x + dx]) - c) > t
            fn, fe, fs, fw = d(0, -3), d(3, 0), d(0, 3), d(-3, 0)
            if eight:
                f = [fn, d(2, -2), fe, d(2, 2), fs, d(-2, 2), fw, d(-2, -2)]
                out[(i, col)] = any(all(f[(s + k) % 8] for k in range(4)) for s in range(8))
            elif three:
                out[(i, col)] = fn + fe + fs + fw >= 3
            else:
                out[(i, col)] = (fn or fs) and (fe or fw)
    return out


def test_shared_comparison_coarse_test_matches_the_rule():
    """The per-lane coarse test (each comparison made once and shared by two
    pixels, neighbour words by lane shuffles) keeps exactly the pixels the
    compass / 8-point rules keep, on every column the NMS reads."""
    rng = np.random.default_rng(11)
    rows = 8
    for trial in range(24):
        xoff = 4 if trial % 2 == 0 else 12
        xw = xoff // 4
        # smooth background plus sharp blocks: every flag combination occurs
        box = np.clip(rng.normal(128, 25, (rows + 6, 144)), 0, 255).astype(np.int64)
        for _ in range(12):
            y, x = rng.integers(0, rows + 6), rng.integers(0, 140)
            box[y:y + rng.integers(1, 6), x:x + rng.integers(1, 8)] = rng.integers(0, 256)
        t = [0, 5, 15, 40, 127, 128, 200][trial % 7]
        three = trial % 5 == 4
        eight = not three and trial % 3 != 0
        radius = 1 if trial % 4 < 2 else 2
        got = _coarse_warp(box, xw, t, rows, three, eight, radius)
        want = _coarse_reference(box, xoff, t, rows, three, eight)
        for col in range(4 - radius, 124 + radius):
            for i in range(rows):
                assert got[(i, col)] == want[(i, col)], (trial, i, col, t, three, eight, radius)


def test_prmt_sign_flags_build_the_masks():
    """eval_corner's mask assembly: prmt with sign replication of the label
    words of points i and i + 8, bit i of each byte, a final byte reorder;
    equals the Eq. 1 masks (bright bits 0..15, dark bits 16..31)."""
    def prmt(a, b, sel):
        src = [(a >> (8 * k)) & 0xFF for k in range(4)] + [(b >> (8 * k)) & 0xFF for k in range(4)]
        out = 0
        for k in range(4):
            nib = (sel >> (4 * k)) & 0xF
            byte = src[nib & 7]
            if nib & 8:
                byte = 0xFF if byte & 0x80 else 0
            out |= byte << (8 * k)
        return out
    rng = np.random.default_rng(12)
    for _ in range(20000):
        c, t = int(rng.integers(0, 256)), int(rng.integers(0, 256))
        v = [int(x) if rng.random() < 0.5 else int(np.clip(c + rng.integers(-t - 2, t + 3), 0, 255))
             for x in rng.integers(0, 256, 16)]
        K = ((0x7FFF - c - t) & 0xFFFF) | (((0x7FFF + c - t) & 0xFFFF) << 16)
        w = [(K + x * 0xFFFF0001) & 0xFFFFFFFF for x in v]
        acc = 0
        for i in range(8):
            acc |= prmt(w[i], w[i + 8], 0xFDB9) & (0x01010101 << i)
        acc = prmt(acc, 0, 0x3120)
        want = sum(1 << i for i in range(16) if v[i] > c + t) | (sum(1 << i for i in range(16) if v[i] < c - t) << 16)
        assert acc == want


def test_sweep_window_minima_give_the_segment_test():
    """The sweep's full test: with D_i = (v_i - c + 256) | (c - v_i + 256) << 16,
    minima of three and of eight points, and windows of n = 8 + R as two
    windows of 8 that are R apart, the largest window minimum is >= t + 257
    exactly when the pixel is a corner at threshold t with arc length n."""
    rng = np.random.default_rng(13)
    for trial in range(4000):
        c = int(rng.integers(0, 256))
        v = [int(x) for x in np.clip(c + rng.integers(-60, 61, 16), 0, 255)]
        if trial % 2:
            s0, L, sg = int(rng.integers(0, 16)), int(rng.integers(8, 17)), 1 if rng.random() < 0.5 else -1
            for j in range(L):
                v[(s0 + j) % 16] = int(np.clip(c + sg * rng.integers(1, 90), 0, 255))
        D = [(x - c + 256) | ((c - x + 256) << 16) for x in v]
        lo = lambda w: w & 0xFFFF
        hi = lambda w: w >> 16
        mn = lambda *ws: (min(lo(w) for w in ws)) | (min(hi(w) for w in ws) << 16)
        W3 = [mn(D[i], D[(i + 1) % 16], D[(i + 2) % 16]) for i in range(16)]
        W8 = [mn(W3[i], W3[(i + 3) % 16], W3[(i + 5) % 16]) for i in range(16)]
        for n in range(9, 17):
            Wn = [mn(W8[i], W8[(i + n - 8) % 16]) for i in range(16)]
            best = max(max(lo(w), hi(w)) for w in Wn)
            for t in (0, 5, 10, 20, 40, 100, 255):
                b = sum(1 << i for i in range(16) if v[i] > c + t)
                d = sum(1 << i for i in range(16) if v[i] < c - t)
                assert (best >= t + 257) == (_has_run(b, n) or _has_run(d, n)), (v, c, t, n)



def test_sweep_packed_setting_compares():
    """The sweep's per-setting compares, two settings per word: lane h of
    pair j holds setting 2j + h's threshold + 257 (0x7FFF when unused), a
    byte permute picks each lane's window minimum from best_a (bytes 0-1) or
    best_b (bytes 2-3), and bit 15 of 0x8000 + best - (t + 257) per lane,
    gathered to bit s, equals best >= t + 257 for every setting s."""
    rng = np.random.default_rng(29)
    for trial in range(3000):
        n_set = int(rng.integers(1, 9))
        ts = [int(x) for x in rng.integers(0, 256, n_set)]
        use_b = [bool(x) for x in rng.integers(0, 2, n_set)]
        if trial < 40:
            ts = [0 if trial % 2 else 255] * n_set
        tpair, selp = [], [0, 0]
        for j in range(4):
            pr = sl = 0
            for h in range(2):
                s = 2 * j + h
                pr |= ((ts[s] + 257) if s < n_set else 0x7FFF) << (16 * h)
                sl |= (0x32 if s < n_set and use_b[s] else 0x10) << (8 * h)
            tpair.append(pr)
            selp[j // 2] |= sl << (16 * (j & 1))
        for best_a, best_b in [(int(a), int(b)) for a, b in rng.integers(0, 512, (8, 2))] + [(0, 511), (511, 0), (257, 256)]:
            bb = best_a | (best_b << 16)
            z = 0
            for j in range(4):
                x = (_byte_perm(bb, 0, (selp[j // 2] >> (16 * (j & 1))) & 0xFFFF) + 0x80008000 - tpair[j]) & 0xFFFFFFFF
                z |= (x & 0x80008000) >> (15 - 2 * j)
            cmask = (z | (z >> 15)) & 0xFF
            want = sum(1 << s for s in range(n_set) if (best_b if use_b[s] else best_a) >= ts[s] + 257)
            assert cmask == want, (ts, use_b, best_a, best_b)



def test_two_ended_walk_emits_every_bit_once():
    """The detect kernel's compaction walk: each step takes the highest set
    bit (31 - clz) and the lowest (the isolated bit m & -m), clears both with
    m &= (m - 1) & ~high, and writes the second only when the two differ; the
    written bits are the mask's bits, each once."""
    rng = np.random.default_rng(41)
    masks = [0, 1, 1 << 31, 0xFFFFFFFF, 0x80000001, 0x00010000] + [int(x) for x in rng.integers(0, 2**32, 3000, dtype=np.uint64)]
    masks += [int(x) & int(y) & int(z) for x, y, z in rng.integers(0, 2**32, (2000, 3), dtype=np.uint64)]
    for m in masks:
        out, mw, steps = [], m, 0
        while mw:
            bh = mw.bit_length() - 1
            lowbit = mw & ((-mw) & 0xFFFFFFFF)
            bl = lowbit.bit_length() - 1
            hb = 1 << bh
            mw &= ((mw - 1) & 0xFFFFFFFF) & (~hb & 0xFFFFFFFF)
            out.append(bh)
            if lowbit != hb:
                out.append(bl)
            steps += 1
        assert sorted(out) == [b for b in range(32) if (m >> b) & 1], hex(m)
        assert steps == (bin(m).count("1") + 1) // 2


def test_walk_code_decodes_to_the_pixel():
    """walk_code_index: the raw code w << 10 | lane << 5 | b of the warp whose
    rows start at r0 is score-region pixel (r0 + 8w + (b & 7)) * 128 +
    4 lane + (b >> 3), for every warp, mask word, lane and bit."""
    for r0 in range(0, 128, 4):
        for w in range(4):
            for lane in range(32):
                for b in range(32):
                    code = (w << 10) | (lane << 5) | b
                    idx = ((r0 + (code & 7) + ((code >> 7) & ~7)) << 7) + ((code >> 3) & 0x7F)
                    assert idx == (r0 + 8 * w + (b & 7)) * 128 + 4 * lane + (b >> 3)



def _ring_offsets(k):
    """The offsets ring_max<K> reads: rows -K and K in full, then columns -K
    and K of the rows between."""
    out = []
    for dx in range(-k, k + 1):
        out += [(-k, dx), (k, dx)]
    for dy in range(-k + 1, k):
        out += [(dy, -k), (dy, k)]
    return out


def test_nms_rings_partition_the_window():
    """The wide NMS windows are tested ring by ring (ring 1 on every corner,
    ring k on the survivors of rings 1..k-1): the rings 1..R visit every
    offset of the (2R+1)^2 window except the centre exactly once, so keeping
    a corner that passes every ring is the plain window test."""
    for r in range(1, 5):
        seen = [o for k in range(1, r + 1) for o in _ring_offsets(k)]
        assert len(seen) == len(set(seen)) == (2 * r + 1) ** 2 - 1
        assert set(seen) == {(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1)} - {(0, 0)}
        for k in range(1, r + 1):
            assert all(max(abs(dy), abs(dx)) == k for dy, dx in _ring_offsets(k))
    rng = np.random.default_rng(47)
    for _ in range(200):
        r = int(rng.integers(2, 5))
        tile = rng.integers(0, 6, (2 * r + 1, 2 * r + 1))
        s = tile[r, r]
        window = all(s >= tile[r + dy, r + dx] for dy in range(-r, r + 1) for dx in range(-r, r + 1))
        rings = all(all(s >= tile[r + dy, r + dx] for dy, dx in _ring_offsets(k)) for k in range(1, r + 1))
        assert window == rings



def test_sweep_first_pass_keeps_every_setting():
    """The sweep's first pass tests the lowest threshold and the shortest
    arc length of the launch: a pixel that is a corner at (t, n) with
    t >= t_min and n >= n_min is one at (t_min, n_min)."""
    rng = np.random.default_rng(43)
    for trial in range(3000):
        c = int(rng.integers(0, 256))
        v = [int(x) for x in np.clip(c + rng.integers(-70, 71, 16), 0, 255)]
        if trial % 2:
            s0, L, sg = int(rng.integers(0, 16)), int(rng.integers(9, 17)), 1 if rng.random() < 0.5 else -1
            for j in range(L):
                v[(s0 + j) % 16] = int(np.clip(c + sg * rng.integers(1, 90), 0, 255))

        def corner(t, n):
            b = sum(1 << i for i in range(16) if v[i] > c + t)
            d = sum(1 << i for i in range(16) if v[i] < c - t)
            return _has_run(b, n) or _has_run(d, n)

        t_min, n_min = int(rng.integers(0, 60)), int(rng.integers(9, 17))
        for t in (t_min, t_min + 1, t_min + 7, t_min + 40, 255):
            for n in range(n_min, 17):
                if corner(t, n):
                    assert corner(t_min, n_min), (v, c, t, n, t_min, n_min)



def test_row_flag_accumulation_and_masks():
    """coarse_and_compact's candidate words: each row's flags (bit 7 of each
    byte) enter at the top and shift down one bit per row, so bit 8j + i of
    word w is row 8w + i, column j; a last word of fewer than 8 rows is
    shifted down; rows outside [row_lo, row_hi) and masked columns are
    cleared at the end.  Decoding the set bits gives exactly the kept pixels."""
    rng = np.random.default_rng(15)
    for _ in range(5000):
        rpw = int(rng.choice([4, 8, 16]))
        r0 = rpw * int(rng.integers(0, 8))
        lane = int(rng.integers(0, 32))
        keeps = [int(x) for x in rng.integers(0, 1 << 32, rpw, dtype=np.uint64)]
        vmb = int(rng.integers(0, 16))
        vm = sum(0x80 << (8 * j) for j in range(4) if (vmb >> j) & 1)
        row_lo, row_hi = int(rng.integers(-3, 70)), int(rng.integers(-3, 70))
        nw = (4 * rpw + 31) // 32
        m = [0] * nw
        for i in range(rpw):
            m[i // 8] = (m[i // 8] >> 1) | (keeps[i] & 0x80808080)
        if rpw % 8:
            m[nw - 1] >>= 8 - rpw % 8
        cols = ((vm >> 7) & 0x01010101) * 0xFF
        for w in range(nw):
            lo = min(max(row_lo - r0 - 8 * w, 0), 8)
            hi = min(max(row_hi - r0 - 8 * w, 0), 8)
            m[w] &= ((((0xFF << lo) & ~(0xFF << hi)) & 0xFF) * 0x01010101) & cols
        got = {(r0 + 8 * w) * 128 + 4 * lane + (b & 7) * 128 + (b >> 3)
               for w in range(nw) for b in range(32) if (m[w] >> b) & 1}
        want = {(r0 + i) * 128 + 4 * lane + j for i in range(rpw) for j in range(4)
                if row_lo <= r0 + i < row_hi and (keeps[i] >> (8 * j + 7)) & 1 and (vmb >> j) & 1}
        assert got == want


def test_pyramid_block_row_by_multiply_high():
    """pyramid_kernel's block row: umulhi(2 * block, ceil(2^31 / pyr_bx))
    equals block / pyr_bx for every block index below 2^16 and every
    pyr_bx up to 256 (frames up to 131072 pixels wide; the ABI allows 65535)."""
    for bx in range(1, 257):
        m = ((1 << 31) + bx - 1) // bx
        assert m < (1 << 32)
        lb = np.arange(1 << 16, dtype=np.uint64)
        assert np.array_equal(((2 * lb) * np.uint64(m)) >> np.uint64(32), lb // np.uint64(bx))


def test_pair_sums_odd_bytes_by_byte_permute():
    """pair_sums: __byte_perm(w, 0, 0x4341) moves bytes 1 and 3 into the low
    halves of the 16-bit lanes, i.e. (w >> 8) & 0x00FF00FF."""
    rng = np.random.default_rng(16)
    for w in [int(x) for x in rng.integers(0, 1 << 32, 20000, dtype=np.uint64)] + [0, 0xFFFFFFFF]:
        assert _byte_perm(w, 0, 0x4341) == (w >> 8) & 0x00FF00FF
