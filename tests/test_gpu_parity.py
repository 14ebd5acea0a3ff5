"""GPU parity: the CUDA path (called through the C ABI) against the CPU
oracle, element by element, bit-exact (integer arithmetic throughout)."""
import numpy as np
import pytest

import oracle
from paper_2003_13493_gb300 import synth, vio

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dets():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    out = {m: vio.Detector(device=0, max_frames=64, score=m) for m in (0, 1, 2)}
    yield out
    for d in out.values():
        d.close()


def to_gpu(img, pitch=None, offset=0):
    """Device copy of img with row pitch `pitch` and base offset `offset` bytes."""
    h, w = img.shape
    pitch = pitch or w
    buf = torch.zeros(h * pitch + offset + 64, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + h * pitch].view(h, pitch)[:, :w]
    view.copy_(torch.from_numpy(img).cuda())
    return view


def run(det, imgs, thresh, arc, cell, levels, **kw):
    frames = [to_gpu(im, **kw) for im in imgs]
    outs, counts = det.detect(frames, thresh, arc, cell, levels)
    det.sync()
    return [o.cpu().numpy() for o in outs], counts.cpu().numpy()


def assert_parity(got, counts, imgs, thresh, arc, cell, levels, mode, nms_radius=1):
    for i, img in enumerate(imgs):
        want, n = oracle.detect(img, thresh, arc, cell, levels, mode, nms_radius=nms_radius)
        if not np.array_equal(got[i], want):
            bad = np.nonzero((got[i] != want).any(axis=1))[0]
            raise AssertionError(f"frame {i} ({img.shape[1]}x{img.shape[0]}): {len(bad)} cells differ, "
                                 f"first {bad[:3].tolist()}: got {got[i][bad[:3]].tolist()} "
                                 f"want {want[bad[:3]].tolist()}")
        assert counts[i] == n, (i, counts[i], n)


# ---- the five workloads ----------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1, 2])
def test_single_frame_one_level(dets, mode):
    img = synth.make_frame(752, 480, seed=0)
    got, cnt = run(dets[mode], [img], 10, 9, 32, 1)
    assert_parity(got, cnt, [img], 10, 9, 32, 1, mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_single_frame_three_levels(dets, mode):
    img = synth.make_frame(752, 480, seed=1)
    got, cnt = run(dets[mode], [img], 20, 9, 32, 3)
    assert_parity(got, cnt, [img], 20, 9, 32, 3, mode)


@pytest.fixture(scope="module")
def mixed():
    return synth.mixed_batch(first_seed=2, per_size=16)


@pytest.mark.parametrize("cell", [32, 64])
def test_mixed_batch_64_frames(dets, mixed, cell):
    got, cnt = run(dets[0], mixed, 15, 9, cell, 3)
    assert_parity(got, cnt, mixed, 15, 9, cell, 3, 0)


SWEEP = [(t, a) for a in (12, 9) for t in (5, 10, 20, 40)]


def test_large_frames_sweep_pyramid_once(dets):
    """3840x2160, 4 levels, 64x64 cells, the 8 (thresh, arc) settings in one
    sweep call (pyramid built once): every setting equals a plain vio_detect
    call; frame 0 is checked against the oracle for all settings, frame 1 for
    one."""
    imgs = [synth.make_frame(3840, 2160, seed=100 + i, n_shapes=400) for i in range(2)]
    frames = [to_gpu(im) for im in imgs]
    outs, counts = dets[0].detect_sweep(frames, SWEEP, 64, 4)
    dets[0].sync()
    cnt = counts.cpu().numpy()
    for p, (thresh, arc) in enumerate(SWEEP):
        got = [o.cpu().numpy() for o in outs[p]]
        ref, ref_cnt = run(dets[0], imgs, thresh, arc, 64, 4)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), (thresh, arc)
        assert np.array_equal(cnt[p], ref_cnt)
        check = imgs if (thresh, arc) == (10, 9) else imgs[:1]
        assert_parity(got, cnt[p], check, thresh, arc, 64, 4, 0)


# settings out of threshold order, repeated thresholds, one at or above 128,
# every arc length, more than the 8 settings one fused launch takes
SWEEP_WIDE = [(40, 9), (5, 12), (20, 16), (5, 9), (130, 9), (12, 10), (12, 11), (20, 13), (7, 14), (60, 15)]


def test_fused_sweep_groups_orders_and_fallbacks(dets, mixed):
    imgs = mixed[::7]
    frames = [to_gpu(im) for im in imgs]
    outs, counts = dets[0].detect_sweep(frames, SWEEP_WIDE, 32, 3)
    dets[0].sync()
    cnt = counts.cpu().numpy()
    for p, (thresh, arc) in enumerate(SWEEP_WIDE):
        got = [o.cpu().numpy() for o in outs[p]]
        assert_parity(got, cnt[p], imgs, thresh, arc, 32, 3, 0)
    # contexts the fused launch does not serve (MT score, 5x5 NMS) run one
    # detection per setting and must agree with the oracle all the same
    wide = vio.Detector(max_frames=16, nms_radius=2)
    for det, mode, radius in ((dets[2], 2, 1), (wide, 0, 2)):
        o2, c2 = det.detect_sweep(frames[:3], SWEEP_WIDE[:3], 32, 3)
        det.sync()
        for p, (thresh, arc) in enumerate(SWEEP_WIDE[:3]):
            assert_parity([o.cpu().numpy() for o in o2[p]], c2.cpu().numpy()[p], imgs[:3], thresh, arc, 32, 3,
                          mode, nms_radius=radius)
    wide.close()


def test_large_frames_sampled(dets):
    """3840x2160, 4 levels, 64x64 cells: two frames of the 32-frame set in
    one launch, all eight (arc, thresh) combinations checked on frame 0 and
    one combination on frame 1."""
    imgs = [synth.make_frame(3840, 2160, seed=100 + i, n_shapes=400) for i in range(2)]
    frames = [to_gpu(im) for im in imgs]
    for arc in (12, 9):
        for thresh in (5, 10, 20, 40):
            outs, counts = dets[0].detect(frames, thresh, arc, 64, 4)
            dets[0].sync()
            got = [o.cpu().numpy() for o in outs]
            cnt = counts.cpu().numpy()
            check = imgs if (arc, thresh) == (9, 10) else imgs[:1]
            assert_parity(got, cnt, check, thresh, arc, 64, 4, 0)


def cells_from_oracle_crop(img, ox, oy, cw, ch, thresh, arc, cell, levels, mode=0):
    """Records of the cells [ox, ox + cw) x [oy, oy + ch) (level-0 pixels, on
    the cell grid) of a frame too large for the oracle, computed by the oracle
    on a crop: every level's score map and 3x3 NMS on the crop's pyramid, then
    the cell maxima (highest score, then lower level, y, x) over the
    survivors inside each cell.  The crop starts 4 pixels of the coarsest
    level before the cells (aligned to 2^(levels-1)) and ends as far after
    them, so the circle and NMS context of every pixel in the cells is in it."""
    h, w = img.shape
    a = 1 << (levels - 1)
    m = 4 * a
    x0, y0 = max(0, ox - m), max(0, oy - m)
    x1, y1 = min(w, ox + cw + m), min(h, oy + ch + m)
    x1 = x0 + (x1 - x0) // a * a if x1 < w else x1
    y1 = y0 + (y1 - y0) // a * a if y1 < h else y1
    crop = np.ascontiguousarray(img[y0:y1, x0:x1])
    gx, gy = (cw + cell - 1) // cell, (ch + cell - 1) // cell
    best = {}
    for k, lev in enumerate(oracle.pyramid(crop, levels)):
        surv = oracle.nms(oracle.score_map(lev, thresh, arc, mode), 1)
        ys, xs = np.nonzero(surv)
        for yk, xk in zip(ys, xs):
            X, Y = ((int(xk) + (x0 >> k)) << k), ((int(yk) + (y0 >> k)) << k)
            if not (ox <= X < ox + cw and oy <= Y < oy + ch):
                continue
            cid = ((Y - oy) // cell) * gx + (X - ox) // cell
            key = (int(surv[yk, xk]), -k, -(int(yk) + (y0 >> k)), -(int(xk) + (x0 >> k)))
            if cid not in best or key > best[cid][0]:
                best[cid] = (key, (X, Y, k, int(surv[yk, xk])))
    out = np.tile(np.array([-1, -1, -1, 0], np.int32), (gx * gy, 1))
    for cid, (_, rec) in best.items():
        out[cid] = rec
    return out


def test_maximum_frame_size_sampled(dets):
    """The largest frame the ABI takes (w * h just below 2^28), 3 levels, 64x64
    cells: 16 blocks of 3x3 cells (corners, edges, interior) against the
    oracle on crops; the next larger frame is rejected."""
    base = synth.make_frame(2048, 2048, seed=123, n_shapes=60)
    W, H = 16384, 16383
    img = np.ascontiguousarray(np.tile(base, (8, 8))[:H, :W])
    frame = to_gpu(img)
    outs, counts = dets[0].detect([frame], 15, 9, 64, 3)
    dets[0].sync()
    got = outs[0].cpu().numpy()
    gw = (W + 63) // 64
    gh = (H + 63) // 64
    rng = np.random.default_rng(3)
    blocks = [(0, 0), (gw - 3, 0), (0, gh - 3), (gw - 3, gh - 3)]
    blocks += [(int(rng.integers(0, gw - 3)), int(rng.integers(0, gh - 3))) for _ in range(12)]
    for bx, by in blocks:
        ox, oy = bx * 64, by * 64
        cw, ch = min(3 * 64, W - ox), min(3 * 64, H - oy)
        want = cells_from_oracle_crop(img, ox, oy, cw, ch, 15, 9, 64, 3)
        ncx = (cw + 63) // 64
        for j in range((ch + 63) // 64):
            for i in range(ncx):
                assert np.array_equal(got[(by + j) * gw + bx + i], want[j * ncx + i]), (bx + i, by + j)
    assert counts.cpu().numpy()[0] == int((got[:, 2] >= 0).sum())
    too_big = torch.zeros((16384, 16384), dtype=torch.uint8, device="cuda")
    with pytest.raises(vio.VioError):
        dets[0].detect([too_big], 15, 9, 64, 3)


@pytest.mark.parametrize("levels", [1, 2])
def test_width_limit(dets, levels):
    """Frames at the width limit: level x coordinates close to 2^16, where
    the cell index of a level pixel (a multiply-high by ceil(2^32 / C_k)) is
    still exact; a frame one pixel wider is rejected."""
    W, H = 65528, 64
    base = synth.make_frame(4096, 64, seed=321, n_shapes=24)
    img = np.ascontiguousarray(np.tile(base, (1, 16))[:, :W])
    got, cnt = run(dets[0], [img], 15, 9, 32, levels)
    assert_parity(got, cnt, [img], 15, 9, 32, levels, 0)
    # the last column of cells has features: x near 2^16 is exercised
    last = got[0].reshape(-1, (W + 31) // 32, 4)[:, -4:]
    assert (last[..., 2] >= 0).any()
    for w in (65535, 65536):
        frame = torch.zeros((16, w), dtype=torch.uint8, device="cuda")
        if w <= 65535:
            dets[0].detect([frame], 15, 9, 32, 1)
            dets[0].sync()
        else:
            with pytest.raises(vio.VioError):
                dets[0].detect([frame], 15, 9, 32, 1)


def test_large4k_sweep_full_launch_sampled(dets):
    """The 4K sweep exactly as the benchmark launches it: all 32 frames of
    3840x2160 (seeds 100..131, 400 shapes), 4 levels, 64x64 cells, the 8
    (thresh, arc) settings in one fused sweep.  Every frame and setting is
    checked on two blocks of 3x3 cells against the oracle on crops, and the
    counts against the records."""
    imgs = [synth.make_frame(3840, 2160, seed=100 + i, n_shapes=400) for i in range(32)]
    frames = [to_gpu(im) for im in imgs]
    outs, counts = dets[0].detect_sweep(frames, SWEEP, 64, 4)
    dets[0].sync()
    cnt = counts.cpu().numpy()
    gw, gh = 60, 34
    rng = np.random.default_rng(11)
    for i, im in enumerate(imgs):
        blocks = [(int(rng.integers(0, gw - 3)), int(rng.integers(0, gh - 3))) for _ in range(2)]
        for p, (thresh, arc) in enumerate(SWEEP):
            got = outs[p][i].cpu().numpy()
            assert cnt[p][i] == int((got[:, 2] >= 0).sum())
            for bx, by in blocks:
                ox, oy = bx * 64, by * 64
                cw, ch = min(192, 3840 - ox), min(192, 2160 - oy)
                want = cells_from_oracle_crop(im, ox, oy, cw, ch, thresh, arc, 64, 4)
                ncx = (cw + 63) // 64
                for j in range((ch + 63) // 64):
                    for k in range(ncx):
                        assert np.array_equal(got[(by + j) * gw + bx + k], want[j * ncx + k]), (i, p, bx + k, by + j)


# ---- edge cases -------------------------------------------------------------

EDGE_SIZES = [(7, 7, 1), (8, 7, 1), (13, 9, 1), (31, 17, 1), (100, 37, 2), (257, 131, 3),
              (640, 480, 4), (1920, 1080, 5), (333, 999, 3), (4000, 70, 3), (56, 56, 3)]


@pytest.mark.parametrize("w,h,levels", EDGE_SIZES)
def test_ragged_sizes(dets, w, h, levels):
    img = synth.make_frame(w, h, seed=w * 1000 + h, n_shapes=10)
    for mode in (0, 1, 2):
        got, cnt = run(dets[mode], [img], 8, 9, 32, levels)
        assert_parity(got, cnt, [img], 8, 9, 32, levels, mode)


def test_pitch_and_alignment_paths(dets):
    img = synth.make_frame(301, 203, seed=4, n_shapes=12)
    for pitch, offset in ((None, 0), (304, 0), (320, 0), (301, 1), (512, 16), (320, 3)):
        got, cnt = run(dets[0], [img], 12, 9, 32, 3, pitch=pitch, offset=offset)
        assert_parity(got, cnt, [img], 12, 9, 32, 3, 0)


@pytest.mark.parametrize("thresh,arc,cell", [(0, 9, 32), (1, 16, 32), (255, 9, 32), (254, 9, 64),
                                             (30, 12, 96), (15, 13, 160), (5, 10, 32)])
def test_parameter_edges(dets, thresh, arc, cell):
    img = synth.make_frame(640, 480, seed=thresh + arc, n_shapes=40)
    modes = (0, 1) if thresh == 0 else (0, 1, 2)
    for mode in modes:
        got, cnt = run(dets[mode], [img], thresh, arc, cell, 3)
        assert_parity(got, cnt, [img], thresh, arc, cell, 3, mode)


def test_degenerate_frames(dets):
    flat = np.full((64, 96), 77, dtype=np.uint8)
    checker = ((np.indices((64, 64)).sum(axis=0) % 2) * 255).astype(np.uint8)
    dot = np.zeros((7, 7), dtype=np.uint8)
    dot[3, 3] = 250
    plateau = np.zeros((40, 40), dtype=np.uint8)
    plateau[10:30, 10:30] = 200  # a square: equal-score corners and ties
    for img in (flat, checker, dot, plateau):
        for mode in (0, 1, 2):
            got, cnt = run(dets[mode], [img], 10, 9, 32, 1)
            assert_parity(got, cnt, [img], 10, 9, 32, 1, mode)
    got, cnt = run(dets[0], [flat], 0, 9, 32, 3)
    assert cnt[0] == 0 and (got[0][:, 2] == -1).all()


# ---- invariance across launch forms ------------------------------------------

def test_every_tile_variant_is_identical(dets, mixed):
    imgs = mixed[::8]
    ref, ref_cnt = run(dets[0], imgs, 15, 9, 32, 3)
    frames = [to_gpu(im) for im in imgs]
    for v in vio.variant_ids(1):
        dets[0].set_variant(v)
        outs, counts = dets[0].detect(frames, 15, 9, 32, 3)
        dets[0].sync()
        for a, b in zip(outs, ref):
            assert np.array_equal(a.cpu().numpy(), b), v
        assert np.array_equal(counts.cpu().numpy(), ref_cnt)
    dets[0].set_variant(None)
    assert_parity(ref, ref_cnt, imgs, 15, 9, 32, 3, 0)


def test_graphs_off_and_autotune_identical(mixed):
    imgs = mixed[::4]
    a = vio.Detector(max_frames=64, use_graphs=False)
    b = vio.Detector(max_frames=64, autotune=True)
    ra, ca = run(a, imgs, 15, 9, 32, 3)
    rb, cb = run(b, imgs, 15, 9, 32, 3)
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    assert np.array_equal(ca, cb)
    assert_parity(ra, ca, imgs, 15, 9, 32, 3, 0)
    a.close()
    b.close()


def test_repeated_calls_and_shape_changes(dets, mixed):
    """Keys are cleared by each call; alternating shapes reuse plans."""
    seq = [(mixed[0:3], 3), (mixed[20:21], 2), (mixed[0:3], 3), (mixed[40:48], 1), (mixed[20:21], 2)]
    for imgs, levels in seq:
        got, cnt = run(dets[0], imgs, 15, 9, 32, levels)
        assert_parity(got, cnt, imgs, 15, 9, 32, levels, 0)


def test_host_path_matches(dets, mixed):
    imgs = mixed[::6]
    outs, counts = dets[0].detect_host(imgs, 15, 9, 32, 3)
    assert_parity(outs, counts, imgs, 15, 9, 32, 3, 0)
    # non-contiguous host rows (pitch > w)
    big = np.zeros((480, 800), dtype=np.uint8)
    big[:, :752] = mixed[16]
    outs, counts = dets[0].detect_host([big[:, :752]], 15, 9, 32, 3)
    assert_parity(outs, counts, [mixed[16]], 15, 9, 32, 3, 0)


def pinned_like(a, offset=0):
    """A page-locked host copy of a (numpy view of pinned torch memory),
    starting `offset` bytes into its buffer."""
    buf = torch.empty(a.nbytes + offset + 64, dtype=torch.uint8).pin_memory()
    v = buf.numpy()[offset:offset + a.nbytes].view(a.dtype).reshape(a.shape)
    v[...] = a
    return buf, v


def test_host_path_pinned_buffers(dets, mixed):
    """Pinned frames are read by the pyramid kernel through their device
    mapping and pinned outputs are written in place; the results must not
    change, alone or mixed with pageable and misaligned buffers."""
    imgs = mixed[::6]
    keep = []
    frames = []
    for i, im in enumerate(imgs):
        if i % 3 == 0:
            frames.append(im)                         # pageable: copy engine
        else:
            b, v = pinned_like(im, offset=0 if i % 3 == 1 else 1)  # aligned / misaligned pinned
            keep.append(b)
            frames.append(v)
    outs = []
    for i, im in enumerate(imgs):
        shape = (vio.num_cells(im.shape[1], im.shape[0], 32), 4)
        if i % 2:
            b, v = pinned_like(np.full(shape, 7, np.int32))
            keep.append(b)
            outs.append(v)
        else:
            outs.append(np.full(shape, 7, np.int32))
    for mode in (0, 2):
        got, counts = dets[mode].detect_host(frames, 15, 9, 32, 3, outs=outs)
        assert_parity(got, counts, imgs, 15, 9, 32, 3, mode)
    # one level: no pyramid kernel, the pinned frames take the copy engine
    got, counts = dets[0].detect_host(frames, 15, 9, 32, 1, outs=[np.empty_like(o) for o in outs])
    assert_parity(got, counts, imgs, 15, 9, 32, 1, 0)


def arena_frames(imgs, layout, pinned=True):
    """Frames placed in one host buffer: layout[i] = (gap bytes before frame
    i, row pitch or 0 for w).  Returns the buffer and numpy views."""
    spans = []
    off = 0
    for im, (gap, pitch) in zip(imgs, layout):
        h, w = im.shape
        pitch = pitch or w
        off += gap
        spans.append((off, pitch))
        off += pitch * (h - 1) + w
    buf = torch.zeros(off + 64, dtype=torch.uint8)
    if pinned:
        buf = buf.pin_memory()
    a = buf.numpy()
    views = []
    for im, (o, pitch) in zip(imgs, spans):
        h, w = im.shape
        v = np.lib.stride_tricks.as_strided(a[o:], shape=(h, w), strides=(pitch, 1))
        v[...] = im
        views.append(v)
    return buf, views


def test_host_frames_in_one_buffer(dets, mixed):
    """Frames that lie one after another in host memory are uploaded as
    spans (one copy each); gaps, padded rows, a misaligned frame, a large gap
    and a frame below its predecessor split the spans.  Every layout, pinned
    or pageable, synchronous or pipelined, must give the oracle's records."""
    imgs = [mixed[i] for i in (0, 17, 33, 50, 5, 21, 40, 60)]
    layouts = {
        "packed": [(0, 0)] * len(imgs),
        "gaps and padded rows": [(0, 0), (48, 768), (16, 0), (0, 1936), (4096, 0), (32, 1280), (0, 0), (0, 2048)],
        "misaligned and far": [(0, 0), (0, 0), (3, 0), (13, 0), (8192, 0), (0, 0), (16, 0), (0, 0)],
    }
    for name, layout in layouts.items():
        for pinned in (True, False):
            buf, frames = arena_frames(imgs, layout, pinned)
            got, counts = dets[0].detect_host(frames, 15, 9, 32, 3)
            assert_parity(got, counts, imgs, 15, 9, 32, 3, 0)
            if pinned:
                outs = []
                keep = []
                for im in imgs:
                    b, v = pinned_like(np.zeros((vio.num_cells(im.shape[1], im.shape[0], 32), 4), np.int32))
                    keep.append(b)
                    outs.append(v)
                b, c = pinned_like(np.zeros(len(imgs), np.int32))
                keep.append(b)
                dets[0].detect_host_async(frames, 15, 9, 32, 3, outs, c)
                dets[0].sync()
                assert_parity(outs, c, imgs, 15, 9, 32, 3, 0)
    # frames in reverse address order: every frame its own span
    buf, frames = arena_frames(imgs, layouts["packed"])
    got, counts = dets[0].detect_host(frames[::-1], 15, 9, 32, 3)
    assert_parity(got, counts, imgs[::-1], 15, 9, 32, 3, 0)
    # one level: no pyramid kernel
    got, counts = dets[0].detect_host(frames, 15, 9, 32, 1)
    assert_parity(got, counts, imgs, 15, 9, 32, 1, 0)


def test_host_batch_reuses_marshalled_buffers(dets, mixed):
    """A HostBatch is marshalled once; each call reads the frames' current
    contents (rewritten between calls) and writes the records in place."""
    first = [mixed[i] for i in (1, 18, 35, 52)]
    second = [mixed[i] for i in (9, 26, 43, 60)]  # same sizes, other content
    keep = []
    buf, frames = arena_frames(first, [(0, 0)] * 4)
    outs = []
    for im in first:
        b, v = pinned_like(np.zeros((vio.num_cells(im.shape[1], im.shape[0], 32), 4), np.int32))
        keep.append(b)
        outs.append(v)
    b, counts = pinned_like(np.zeros(4, np.int32))
    keep.append(b)
    batch = vio.HostBatch(frames, outs, counts)
    for imgs in (first, second, first):
        for f, im in zip(frames, imgs):
            f[...] = im
        dets[0].detect_host_batch(batch, 15, 9, 32, 3)
        assert_parity(outs, counts, imgs, 15, 9, 32, 3, 0)
        dets[0].detect_host_batch(batch, 15, 9, 32, 3, pipelined=True)
        dets[0].sync()
        assert_parity(outs, counts, imgs, 15, 9, 32, 3, 0)


def test_host_async_pipelined_on_two_streams(dets, mixed):
    """Batches alternate between two streams with rotating input slots; every
    batch's records must equal the oracle once its stream is synchronised."""
    sets = [mixed[0:16:5], mixed[16:32:5], mixed[32:48:5], mixed[48:64:5]]
    keep = []

    def pinned_outs(imgs):
        outs = []
        for im in imgs:
            b, v = pinned_like(np.zeros((vio.num_cells(im.shape[1], im.shape[0], 32), 4), np.int32))
            keep.append(b)
            outs.append(v)
        b, c = pinned_like(np.zeros(len(imgs), np.int32))
        keep.append(b)
        return outs, c

    frames = []
    for imgs in sets:
        fr = []
        for im in imgs:
            b, v = pinned_like(im)
            keep.append(b)
            fr.append(v)
        frames.append(fr)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    results = []
    for rep in range(2):
        for k, imgs in enumerate(sets):
            outs, counts = pinned_outs(imgs)
            dets[0].detect_host_async(frames[k], 15, 9, 32, 3, outs, counts, stream=streams[k % 2])
            results.append((imgs, outs, counts))
    for st in streams:
        dets[0].sync(st)
    for imgs, outs, counts in results:
        assert_parity(outs, counts, imgs, 15, 9, 32, 3, 0)
    # pageable outputs cannot be written by the device
    with pytest.raises(vio.VioError):
        dets[0].detect_host_async(frames[0], 15, 9, 32, 3, [np.zeros_like(o) for o in results[0][1]])


def test_invalid_arguments_rejected(dets):
    img = to_gpu(synth.make_frame(64, 64, seed=1))
    d = dets[0]
    # cell 0 asks the context to pick the cell size (valid); negative or
    # non-multiples of 32 are not
    bad = [dict(thresh=-1), dict(thresh=256), dict(arc_len=8), dict(arc_len=17), dict(cell=-32),
           dict(cell=48), dict(levels=0), dict(levels=6), dict(levels=4)]  # 64>>3 = 8 ok, 64>>4 < 7
    base = dict(thresh=10, arc_len=9, cell=32, levels=1)
    for b in bad[:-1]:
        kw = {**base, **b}
        with pytest.raises(vio.VioError) as e:
            d.detect([img], kw["thresh"], kw["arc_len"], kw["cell"], kw["levels"])
        assert e.value.status == 1, b
    d.detect([img], 10, 9, 32, 4)  # 8x8 smallest level is fine
    with pytest.raises(vio.VioError):
        d.detect([img], 10, 9, 32, 5)
    with pytest.raises(vio.VioError):
        dets[2].detect([img], 0, 9, 32, 1)  # MT needs thresh >= 1
    small = to_gpu(np.zeros((6, 30), dtype=np.uint8))
    with pytest.raises(vio.VioError):
        d.detect([small], 10, 9, 32, 1)
    d.sync()


def test_budget_exceeded_reports_oom(mixed):
    d = vio.Detector(max_frames=64, mem_budget_bytes=1 << 20)
    frames = [to_gpu(im) for im in mixed[48:64]]
    with pytest.raises(vio.VioError) as e:
        d.detect(frames, 15, 9, 32, 3)
    assert e.value.status == 2
    # a small request still fits the budget afterwards
    outs, counts = d.detect([to_gpu(mixed[0])], 15, 9, 32, 1)
    d.sync()
    want, n = oracle.detect(mixed[0], 15, 9, 32, 1)
    assert np.array_equal(outs[0].cpu().numpy(), want)
    d.close()


def test_alternating_buffers_and_variants(dets):
    """Same batch shape, different frame buffers (and contents) and tile
    variants call after call: every call must read its own frames through
    freshly written tensor maps."""
    a = [synth.make_frame(640, 480, seed=500 + i, n_shapes=30) for i in range(3)]
    b = [synth.make_frame(640, 480, seed=600 + i, n_shapes=30) for i in range(3)]
    ga = [to_gpu(im) for im in a]
    gb = [to_gpu(im) for im in b]
    want_a = [oracle.detect(im, 15, 9, 32, 3)[0] for im in a]
    want_b = [oracle.detect(im, 15, 9, 32, 3)[0] for im in b]
    ids = vio.variant_ids(1)
    nv = len(ids)
    for rep in range(3 * nv):
        dets[0].set_variant(ids[rep % nv] if rep >= nv else None)
        imgs, want = (ga, want_a) if rep % 2 == 0 else (gb, want_b)
        outs, _ = dets[0].detect(imgs, 15, 9, 32, 3)
        dets[0].sync()
        for o, w in zip(outs, want):
            assert np.array_equal(o.cpu().numpy(), w), rep
    dets[0].set_variant(None)


# ---- NMS windows of radius 2..4 (Section I-B, Table III) -----------------------

@pytest.fixture(scope="module")
def wide():
    out = {r: vio.Detector(device=0, max_frames=64, nms_radius=r) for r in (2, 3, 4)}
    yield out
    for d in out.values():
        d.close()


@pytest.mark.parametrize("radius", [2, 3, 4])
def test_wide_nms_mixed_batch(wide, mixed, radius):
    imgs = mixed[::4]
    got, cnt = run(wide[radius], imgs, 15, 9, 32, 3)
    assert_parity(got, cnt, imgs, 15, 9, 32, 3, 0, nms_radius=radius)
    # a wider window never keeps more cells than the 3x3 one finds features in
    want3 = [oracle.detect(im, 15, 9, 32, 3)[1] for im in imgs]
    assert all(c <= w for c, w in zip(cnt, want3))


@pytest.mark.parametrize("radius", [2, 4])
@pytest.mark.parametrize("mode", [1, 2])
def test_wide_nms_other_scores(mode, radius):
    det = vio.Detector(max_frames=4, score=mode, nms_radius=radius)
    img = synth.make_frame(752, 480, seed=31)
    got, cnt = run(det, [img], 12, 9, 32, 3)
    assert_parity(got, cnt, [img], 12, 9, 32, 3, mode, nms_radius=radius)
    det.close()


@pytest.mark.parametrize("radius", [2, 3, 4])
def test_wide_nms_ragged_and_tile_edges(wide, radius):
    # heights around multiples of the tile height (64 - 2r rows) and widths
    # around the 120-pixel tile width, so the window straddles tile seams
    th = 64 - 2 * radius
    sizes = [(7, 7, 1), (31, 17, 1), (121, th + 1, 2), (239, 2 * th - 1, 2), (241, 3 * th, 3), (257, 131, 3)]
    imgs = [synth.make_frame(w, h, seed=900 + i, n_shapes=12) for i, (w, h, _) in enumerate(sizes)]
    for img, (_, _, levels) in zip(imgs, sizes):
        got, cnt = run(wide[radius], [img], 8, 9, 32, levels)
        assert_parity(got, cnt, [img], 8, 9, 32, levels, 0, nms_radius=radius)


def test_wide_nms_autotune_and_tuning(mixed):
    imgs = mixed[::8]
    det = vio.Detector(max_frames=64, nms_radius=3, autotune=True)
    got, cnt = run(det, imgs, 15, 9, 64, 3)
    assert_parity(got, cnt, imgs, 15, 9, 64, 3, 0, nms_radius=3)
    assert det.config().nms_radius == 3
    tw, th, v = det.tuning()
    assert v in vio.variant_ids(3) and th + 6 == 64
    # a variant built for another radius is refused
    with pytest.raises(vio.VioError):
        det.set_variant(vio.variant_ids(1)[0])
    det.close()


def test_autotuner_picks_variant_ctas_and_cell(mixed):
    """cell_size 0 with autotune on: the tuner times every variant x CTAs
    per SM x cell size (32, 64) on the batch, keeps the fastest, and the
    records equal the oracle's at the cell size it reports."""
    imgs = mixed[::4]
    frames = [to_gpu(im) for im in imgs]
    det = vio.Detector(max_frames=64, autotune=True)
    outs = [torch.full((vio.num_cells(im.shape[1], im.shape[0], 32), 4), 7, dtype=torch.int32, device="cuda")
            for im in imgs]
    outs, counts = det.detect(frames, 15, 9, 0, 3, outs=outs)
    det.sync()
    t = det.tuning_full()
    assert t["cell_size"] in (32, 64) and 1 <= t["cta_per_sm"] <= 4 and t["variant"] in vio.variant_ids(1)
    log = det.autotune_log()
    combos = {(e["variant"], e["cta_per_sm"], e["cell_size"]) for e in log}
    assert {e["cell_size"] for e in log} == {32, 64}
    assert {e["cta_per_sm"] for e in log} >= {2, 3}
    assert len(combos) == len(log) >= 2 * len(vio.variant_ids(1))
    best = min(log, key=lambda e: e["ms"])
    assert (best["variant"], best["cta_per_sm"], best["cell_size"]) == (t["variant"], t["cta_per_sm"], t["cell_size"])
    c = t["cell_size"]
    got = [o.cpu().numpy()[:vio.num_cells(im.shape[1], im.shape[0], c)] for o, im in zip(outs, imgs)]
    assert_parity(got, counts.cpu().numpy(), imgs, 15, 9, c, 3, 0)
    # a second call of the same shape reuses the choice without retuning
    det.detect(frames, 15, 9, 0, 3, outs=outs)
    det.sync()
    assert det.tuning_full() == t and len(det.autotune_log()) == len(log)
    det.close()


@pytest.mark.parametrize("ctas", [1, 2, 3, 4])
def test_pinned_ctas_per_sm_identical(dets, mixed, ctas):
    imgs = mixed[::8]
    ref, ref_cnt = run(dets[0], imgs, 15, 9, 32, 3)
    dets[0].set_variant(vio.variant_ids(1)[0], cta_per_sm=ctas)
    got, cnt = run(dets[0], imgs, 15, 9, 32, 3)
    assert dets[0].tuning_full()["cta_per_sm"] == ctas
    dets[0].set_variant(None)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert np.array_equal(cnt, ref_cnt)
    with pytest.raises(vio.VioError):
        dets[0].set_variant(vio.variant_ids(1)[0], cta_per_sm=5)


# ---- the pyramid levels, read back from the context ----

@pytest.mark.parametrize("levels", [2, 3])
def test_pyramid_levels_of_a_batch_match_the_oracle(dets, mixed, levels):
    """The pyramid kernel over a large batch of mixed sizes (odd widths and
    heights included): every pixel of every level equals the oracle's
    pyramid, and so does the detection."""
    imgs = mixed[::3] + [synth.make_frame(643, 479, seed=77), synth.make_frame(1283, 723, seed=78)]
    got, cnt = run(dets[0], imgs, 15, 9, 32, levels)
    for i, img in enumerate(imgs):
        want = oracle.pyramid(img, levels)
        for k in range(1, levels):
            assert np.array_equal(dets[0].copy_level(i, k), want[k]), (i, k, img.shape)
    assert_parity(got, cnt, imgs, 15, 9, 32, levels, 0)


@pytest.mark.parametrize("levels", [3, 4, 5])
def test_pyramid_levels_of_the_pyramid_kernel_match_the_oracle(dets, levels):
    """One frame (a small call: one CTA per SM) at 3 to 5 levels, level 0
    read back as well."""
    img = synth.make_frame(1101, 737, seed=79)
    frame = to_gpu(img, pitch=1120)  # kept alive: level 0 is read back from it
    outs, counts = dets[0].detect([frame], 12, 9, 32, levels)
    dets[0].sync()
    want = oracle.pyramid(img, levels)
    for k in range(levels):
        assert np.array_equal(dets[0].copy_level(0, k), want[k]), k
    assert_parity([outs[0].cpu().numpy()], counts.cpu().numpy(), [img], 12, 9, 32, levels, 0)
    with pytest.raises(vio.VioError):
        dets[0].copy_level(0, levels)
