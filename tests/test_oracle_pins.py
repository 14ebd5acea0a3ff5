"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-derived patterns (tests/golden/fast_patterns.txt), Eq. 1 and the score
  definitions of Section II-D;
* closed forms of the 2x2 half-sampling (Section II-B / III-C);
* an exhaustive check of the arc predicate over all 2^16 label masks
  against the 8 KB bit table of Section II-D built from its definition;
* a second, naive formulation (tests/naive.py) on tiny random images;
* geometric invariants (90-degree rotation, mirror) and monotonicity in the
  threshold and the arc length.
"""
import os

import numpy as np
import pytest

import naive
from paper_2003_13493_gb300.synth import make_frame

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fast_patterns.txt")


def _golden_cases():
    cases, cur = [], None
    with open(GOLDEN) as f:
        lines = [ln.rstrip("\n") for ln in f]
    i = 0
    while i < len(lines):
        ln = lines[i].strip()
        i += 1
        if not ln or ln.startswith("#"):
            continue
        tok = ln.split()
        if tok[0] == "case":
            cur = {"name": tok[1], "checks": [], "grid": []}
        elif tok[0] == "check":
            cur["checks"].append(tuple(int(t) for t in tok[1:]))
        elif tok[0] == "grid":
            while lines[i].strip() != "end":
                cur["grid"].append([int(t) for t in lines[i].split()])
                i += 1
            i += 1
            cases.append(cur)
    return cases


GOLDEN_CASES = _golden_cases()


def test_golden_file_parsed():
    assert len(GOLDEN_CASES) >= 10
    for c in GOLDEN_CASES:
        assert len(c["grid"]) == 7 and all(len(r) == 7 for r in c["grid"]), c["name"]


@pytest.mark.parametrize("case", GOLDEN_CASES, ids=[c["name"] for c in GOLDEN_CASES])
def test_golden_patterns(oracle_mod, case):
    img = np.array(case["grid"], dtype=np.uint8)
    for thresh, arc, corner, sad_b, sad_a, mt in case["checks"]:
        assert oracle_mod.is_corner(img, 3, 3, thresh, arc) == bool(corner), (thresh, arc)
        assert oracle_mod.score_pixel(img, 3, 3, thresh, arc, oracle_mod.SAD_B) == sad_b
        assert oracle_mod.score_pixel(img, 3, 3, thresh, arc, oracle_mod.SAD_A) == sad_a
        assert oracle_mod.score_pixel(img, 3, 3, thresh, arc, oracle_mod.MT) == mt
        # the naive formulation agrees on the hand-derived values too
        g = case["grid"]
        assert naive.score(g, 3, 3, thresh, arc, 0) == sad_b
        assert naive.score(g, 3, 3, thresh, arc, 1) == sad_a
        assert naive.score(g, 3, 3, thresh, arc, 2) == mt


def test_circle_is_bresenham_radius3(oracle_mod):
    # derived independently (midpoint circle construction, angle-sorted)
    assert oracle_mod.circle() == naive.CIRCLE
    assert len(set(naive.CIRCLE)) == 16
    for dx, dy in naive.CIRCLE:
        assert 2.5 <= (dx * dx + dy * dy) ** 0.5 <= 3.5


# ---- pyramid ------------------------------------------------------------


@pytest.mark.parametrize("quad,expect", [((0, 0, 1, 1), 1), ((0, 0, 0, 1), 0), ((1, 2, 2, 2), 2),
                                          ((255, 255, 255, 255), 255), ((0, 0, 0, 0), 0),
                                          ((0, 1, 1, 1), 1), ((3, 3, 3, 2), 3)])
def test_halfsample_closed_form(oracle_mod, quad, expect):
    a, b, c, d = quad
    img = np.array([[a, b], [c, d]], dtype=np.uint8)
    assert oracle_mod.halfsample(img)[0, 0] == expect


def test_halfsample_constant_and_replication(oracle_mod):
    rng = np.random.default_rng(7)
    for v in (0, 17, 128, 255):
        img = np.full((20, 34), v, dtype=np.uint8)
        for lev in oracle_mod.pyramid(img, 4):
            assert (lev == v).all()
    base = rng.integers(0, 256, size=(13, 21), dtype=np.uint8)
    up = np.repeat(np.repeat(base, 2, axis=0), 2, axis=1)
    assert np.array_equal(oracle_mod.halfsample(up), base)
    # odd sizes drop the last row / column
    odd = rng.integers(0, 256, size=(27, 41), dtype=np.uint8)
    hs = oracle_mod.halfsample(odd)
    assert hs.shape == (13, 20)
    assert np.array_equal(hs, naive.pyramid(odd, 2)[1])


# ---- segment test -------------------------------------------------------


def _bit_table(n_arc):
    """The 2^16-entry validity table of Section II-D, one bit per mask
    (word = mask >> 5, bit = mask & 31), built from the definition: a mask is
    valid when its 16 bits hold a cyclic run of n_arc ones."""
    words = np.zeros(2048, dtype=np.uint32)
    for m in range(1 << 16):
        s = format(m, "016b")[::-1]  # bit i -> character i
        if "1" * n_arc in s + s:
            words[m >> 5] |= np.uint32(1) << np.uint32(m & 31)
    return words


@pytest.mark.parametrize("n_arc", list(range(9, 17)))
def test_arc_predicate_exhaustive(oracle_mod, n_arc):
    tab = _bit_table(n_arc)
    assert tab.nbytes == 8192
    lib = oracle_mod._load()
    for m in range(1 << 16):
        want = bool((int(tab[m >> 5]) >> (m & 31)) & 1)
        assert bool(lib.oracle_arc_from_masks(m, 0, n_arc)) == want, (hex(m), n_arc)
        assert bool(lib.oracle_arc_from_masks(0, m, n_arc)) == want, (hex(m), n_arc)


def test_arc_predicate_disjoint_pairs(oracle_mod):
    rng = np.random.default_rng(3)
    lib = oracle_mod._load()
    for _ in range(20000):
        lab = rng.integers(0, 3, size=16)
        b = sum(1 << i for i in range(16) if lab[i] == 1)
        d = sum(1 << i for i in range(16) if lab[i] == 2)
        n = int(rng.integers(9, 17))
        labs = ["b" if v == 1 else ("d" if v == 2 else "s") for v in lab]
        want = naive.has_run(labs, "b", n) or naive.has_run(labs, "d", n)
        assert bool(lib.oracle_arc_from_masks(b, d, n)) == want


# ---- scores: closed forms on generated patterns -------------------------


def _patch(center, vals):
    g = np.full((7, 7), center, dtype=np.uint8)
    for (dx, dy), v in zip(naive.CIRCLE, vals):
        g[3 + dy, 3 + dx] = v
    return g


@pytest.mark.parametrize("k", [9, 10, 12, 15, 16])
@pytest.mark.parametrize("d", [1, 7, 40, 100])
@pytest.mark.parametrize("start", [0, 5, 13])
def test_score_closed_forms(oracle_mod, k, d, start):
    c = 120
    for sign in (+1, -1):
        vals = [c] * 16
        for j in range(k):
            vals[(start + j) % 16] = c + sign * d
        img = _patch(c, vals)
        t = d - 1
        assert oracle_mod.score_pixel(img, 3, 3, t, 9, oracle_mod.SAD_B) == k * d
        assert oracle_mod.score_pixel(img, 3, 3, t, 9, oracle_mod.SAD_A) == k * d
        assert oracle_mod.score_pixel(img, 3, 3, t, 9, oracle_mod.MT) == d - 1
        assert oracle_mod.score_pixel(img, 3, 3, d, 9, oracle_mod.SAD_B) == 0


def test_mt_bruteforce(oracle_mod):
    rng = np.random.default_rng(11)
    hits = 0
    for _ in range(400):
        img = rng.integers(0, 256, size=(7, 7), dtype=np.uint8)
        n = int(rng.integers(9, 13))
        eps = int(rng.integers(1, 60))
        mt = oracle_mod.score_pixel(img, 3, 3, eps, n, oracle_mod.MT)
        brute = max([t for t in range(eps, 256) if oracle_mod.is_corner(img, 3, 3, t, n)], default=0)
        assert mt == brute
        hits += mt > 0
    assert hits > 5


# ---- whole-frame: naive formulation on tiny images ----------------------


def _tiny_images():
    rng = np.random.default_rng(2024)
    out = []
    for i in range(36):
        w = int(rng.integers(7, 41))
        h = int(rng.integers(7, 41))
        kind = i % 3
        if kind == 0:
            img = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
        elif kind == 1:  # few grey levels: many ties and plateaus
            img = (rng.integers(0, 4, size=(h, w)) * 60).astype(np.uint8)
        else:
            img = make_frame(w, h, seed=1000 + i, n_shapes=3)
        out.append(img)
    return out


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_detect_matches_naive_tiny(oracle_mod, mode):
    for i, img in enumerate(_tiny_images()):
        h, w = img.shape
        levels = 1 + (i % 3)
        while levels > 1 and ((w >> (levels - 1)) < 7 or (h >> (levels - 1)) < 7):
            levels -= 1
        cell = 32 if i % 2 else 64
        thresh = [1, 10, 25][i % 3]
        n_arc = 9 + (i % 4)
        got, cnt = oracle_mod.detect(img, thresh, n_arc, cell, levels, mode)
        want = naive.detect(img, thresh, n_arc, cell, levels, mode)
        assert np.array_equal(got, want), (i, w, h, levels)
        assert cnt == int((want[:, 2] >= 0).sum())


def test_score_map_and_nms_match_naive(oracle_mod):
    rng = np.random.default_rng(5)
    for i in range(12):
        h, w = int(rng.integers(7, 30)), int(rng.integers(7, 30))
        img = (rng.integers(0, 6, size=(h, w)) * 40).astype(np.uint8)
        L = img.tolist()
        for mode in (0, 1, 2):
            sm = oracle_mod.score_map(img, 15, 9, mode)
            want = np.array([[naive.score(L, x, y, 15, 9, mode) for x in range(w)] for y in range(h)])
            assert np.array_equal(sm, want)
            assert np.array_equal(oracle_mod.nms3(sm), np.array(naive.nms3(want.tolist())))


# ---- invariants ----------------------------------------------------------


def _nms_maps(oracle_mod, img, thresh, n_arc, levels, mode):
    return [oracle_mod.nms3(oracle_mod.score_map(lev, thresh, n_arc, mode))
            for lev in oracle_mod.pyramid(img, levels)]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_rotation_and_mirror_invariance(oracle_mod, mode):
    img = make_frame(96, 96, seed=77, n_shapes=12)
    base = _nms_maps(oracle_mod, img, 12, 9, 3, mode)
    for op in (lambda a: np.rot90(a, 1), lambda a: np.rot90(a, 2), lambda a: np.rot90(a, 3),
               np.fliplr, np.flipud, np.transpose):
        t = _nms_maps(oracle_mod, np.ascontiguousarray(op(img)), 12, 9, 3, mode)
        for a, b in zip(base, t):
            assert np.array_equal(np.ascontiguousarray(op(a)), b)


def test_cell_output_rotation_for_unique_maxima(oracle_mod):
    img = make_frame(128, 128, seed=5, n_shapes=10)
    cell = 32
    feats, _ = oracle_mod.detect(img, 10, 9, cell, 2)
    rot = np.ascontiguousarray(np.rot90(img, -1))  # clockwise: (x, y) -> (H-1-y, x)
    feats_r, _ = oracle_mod.detect(rot, 10, 9, cell, 2)
    nms = _nms_maps(oracle_mod, img, 10, 9, 2, 0)
    g = 128 // cell
    checked = 0
    for cy in range(g):
        for cx in range(g):
            f = feats[cy * g + cx]
            if f[2] < 0:
                continue
            k = f[2]
            # unique maximum in the cell across levels?
            vals = []
            for lk, m in enumerate(nms):
                c = cell >> lk
                vals.extend(m[cy * c:(cy + 1) * c, cx * c:(cx + 1) * c].ravel().tolist())
            if sorted(vals)[-2] == f[3]:
                continue
            xk, yk = f[0] >> k, f[1] >> k
            wk = 128 >> k
            nx, ny = wk - 1 - yk, xk
            rcx, rcy = (g - 1 - cy), cx
            fr = feats_r[rcy * g + rcx]
            assert (fr[0], fr[1], fr[2], fr[3]) == (nx << k, ny << k, k, f[3])
            checked += 1
    assert checked > 3


def test_threshold_and_arc_monotonicity(oracle_mod):
    img = make_frame(160, 120, seed=9, n_shapes=15)
    prev = None
    for t in (5, 10, 20, 40, 41):
        det = oracle_mod.score_map(img, t, 9, 0) > 0
        if prev is not None:
            assert not (det & ~prev).any()
        prev = det
    prev = None
    for n in range(9, 17):
        det = oracle_mod.score_map(img, 10, n, 0) > 0
        if prev is not None:
            assert not (det & ~prev).any()
        prev = det


def test_conformance_subset_of_plain_fast(oracle_mod):
    """Every selected feature is a plain-FAST corner and a 3x3 local maximum of
    its level (Section III-C conformance: no false positives)."""
    img = make_frame(752, 480, seed=1)
    feats, cnt = oracle_mod.detect(img, 20, 9, 32, 3)
    levels = oracle_mod.pyramid(img, 3)
    assert cnt > 100
    for x, y, k, s in feats:
        if k < 0:
            assert s == 0 and x == -1 and y == -1
            continue
        lev = levels[k]
        xk, yk = x >> k, y >> k
        assert oracle_mod.is_corner(lev, xk, yk, 20, 9)
        assert oracle_mod.score_pixel(lev, xk, yk, 20, 9) == s
        win = oracle_mod.score_map(lev[max(0, yk - 4):yk + 5, max(0, xk - 4):xk + 5], 20, 9)
        assert s > 0
        del win
        nb = [oracle_mod.score_pixel(lev, xk + dx, yk + dy, 20, 9)
              for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        assert s == max(nb)


def test_empty_and_degenerate(oracle_mod):
    flat = np.full((64, 64), 90, dtype=np.uint8)
    feats, cnt = oracle_mod.detect(flat, 0, 9, 32, 3)
    assert cnt == 0 and (feats[:, 2] == -1).all() and (feats[:, 3] == 0).all()
    tiny = np.zeros((7, 7), dtype=np.uint8)
    tiny[3, 3] = 200
    feats, cnt = oracle_mod.detect(tiny, 10, 9, 32, 1)
    assert cnt == 1 and tuple(feats[0]) == (3, 3, 0, 16 * 200)


# ---- larger NMS windows (Section I-B, Table III: n = 2..4) -----------------


@pytest.mark.parametrize("radius", [2, 3, 4])
def test_larger_nms_windows_match_naive(oracle_mod, radius):
    rng = np.random.default_rng(radius)
    for i in range(8):
        h, w = int(rng.integers(7, 30)), int(rng.integers(7, 30))
        img = (rng.integers(0, 5, size=(h, w)) * 50).astype(np.uint8) if i % 2 else \
            make_frame(w, h, seed=300 + i, n_shapes=4)
        sm = oracle_mod.score_map(img, 10, 9, 0)
        assert np.array_equal(oracle_mod.nms(sm, radius), np.array(naive.nms(sm.tolist(), radius)))
        levels = 2 if min(w, h) >= 14 else 1
        got, _ = oracle_mod.detect(img, 10, 9, 32, levels, 0, radius)
        assert np.array_equal(got, naive.detect(img, 10, 9, 32, levels, 0, radius))


def test_nms_windows_nest_and_match_the_3x3_entry(oracle_mod):
    img = make_frame(200, 150, seed=42, n_shapes=12)
    sm = oracle_mod.score_map(img, 12, 9, 0)
    assert np.array_equal(oracle_mod.nms(sm, 1), oracle_mod.nms3(sm))
    prev = oracle_mod.nms(sm, 1) > 0
    for r in (2, 3, 4):
        cur = oracle_mod.nms(sm, r) > 0
        assert not (cur & ~prev).any()  # a wider window only removes survivors
        prev = cur
    # the 3x3 detection equals the default entry point
    a, _ = oracle_mod.detect(img, 12, 9, 32, 2)
    b, _ = oracle_mod.detect(img, 12, 9, 32, 2, 0, 1)
    assert np.array_equal(a, b)
