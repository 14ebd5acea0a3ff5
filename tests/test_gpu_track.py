"""GPU parity of the feature tracker (Section II-E, Eqs. 2-6): the CUDA path
through the C ABI against the fp64 oracle on the same bytes.

Tolerance: the CUDA path computes in fp32.  Both sides iterate Gauss-Newton
to the same fixed point (sum U r = 0), which fp32 moves by far less than the
rounding of a sample position (a level-0 coordinate below 2048 carries an
fp32 rounding error of at most 2^-13 px, i.e. a residual change of gradient
x 1.2e-4 grey and a translation change of ~1e-4 px); positions must agree to
1e-3 px, gain to 1e-4, offset to 2e-2 grey levels and the residual to 1e-3
relative.  The comparison covers the features whose oracle estimate has
converged (it does not move by 1e-6 px with one more iteration on every
level); at least 90 % of the features must be in that set.  Integer outputs
(status, iterations) must match exactly wherever iterations are fixed
(min_update = 0)."""
import numpy as np
import pytest

from oracle import lk_oracle as lk
from paper_2003_13493_gb300 import synth, vio

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

POS_TOL, GAIN_TOL, OFF_TOL, RES_TOL = 1e-3, 1e-4, 2e-2, 1e-3


@pytest.fixture(scope="module")
def det():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    d = vio.Detector(device=0, max_frames=64)
    yield d
    d.close()


def grid(w, h, step, margin):
    ys, xs = np.mgrid[margin:h - margin + 1:step, margin:w - margin + 1:step]
    return np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.float32)


def run(det, pairs, pts, **params):
    prev = [torch.from_numpy(a).cuda() for a, _ in pairs]
    nxt = [torch.from_numpy(b).cuda() for _, b in pairs]
    q = [torch.from_numpy(np.ascontiguousarray(p, dtype=np.float32)).cuda() for p in pts]
    outs = det.track(prev, nxt, q, params)
    det.sync()
    return [o.cpu().numpy() for o in outs]


def oracle_params(params):
    kw = dict(patch_fine=16, patch_coarse=8, max_iters=30, min_update=0.01, model=3)
    kw.update({k: v for k, v in params.items() if k != "levels"})
    return params.get("levels", 3), kw


def converged(prev, nxt, pts, levels, kw):
    """Oracle results and the mask of features whose estimate has converged."""
    a = lk.track(prev, nxt, pts, levels=levels, **kw)
    kw2 = dict(kw, max_iters=kw["max_iters"] + 1)
    b = lk.track(prev, nxt, pts, levels=levels, **kw2)
    ok = (a[:, 4] == b[:, 4]) & (np.abs(a[:, :2] - b[:, :2]).max(axis=1) < 1e-6)
    return a, ok


def assert_close(got, want, mask, exact_iters):
    xy, gain, off, status, iters, res = vio.track_fields(got)
    assert np.array_equal(status[mask], want[mask, 4].astype(np.int32))
    if exact_iters:
        assert np.array_equal(iters[mask], want[mask, 5].astype(np.int32))
    tr = mask & (want[:, 4] == lk.TRACKED)
    assert np.abs(xy[tr] - want[tr, :2]).max(initial=0) < POS_TOL
    assert np.abs(gain[tr] - want[tr, 2]).max(initial=0) < GAIN_TOL
    assert np.abs(off[tr] - want[tr, 3]).max(initial=0) < OFF_TOL
    assert (np.abs(res[tr] - want[tr, 6]) <= RES_TOL * np.maximum(1.0, want[tr, 6])).all()


@pytest.mark.parametrize("model", [0, vio.TRACK_GAIN, vio.TRACK_OFFSET, vio.TRACK_GAIN | vio.TRACK_OFFSET])
def test_models_fixed_iterations(det, model):
    prev = synth.smooth_frame(752, 480, seed=11)
    nxt = synth.smooth_frame(752, 480, seed=11, dx=1.6, dy=-2.3, gain=0.9, offset=8.0)
    pts = grid(752, 480, 37, 40)
    params = dict(levels=3, max_iters=12, min_update=0.0, model=model)
    got = run(det, [(prev, nxt)], [pts], **params)[0]
    L, kw = oracle_params(params)
    want, mask = converged(prev, nxt, pts.astype(np.float64), L, kw)
    assert mask.mean() >= 0.9
    assert_close(got, want, mask, exact_iters=True)


@pytest.mark.parametrize("fine,coarse,levels", [(16, 8, 3), (8, 8, 2), (16, 16, 4), (8, 16, 1)])
def test_patch_sizes_and_levels(det, fine, coarse, levels):
    prev = synth.smooth_frame(640, 480, seed=12)
    nxt = synth.smooth_frame(640, 480, seed=12, dx=-3.2, dy=0.7)
    pts = grid(640, 480, 41, 48)
    params = dict(levels=levels, patch_fine=fine, patch_coarse=coarse, max_iters=15, min_update=0.0, model=3)
    got = run(det, [(prev, nxt)], [pts], **params)[0]
    L, kw = oracle_params(params)
    want, mask = converged(prev, nxt, pts.astype(np.float64), L, kw)
    assert mask.mean() >= 0.9
    assert_close(got, want, mask, exact_iters=True)


def test_default_parameters_with_early_exit(det):
    # the early exit compares |dt| with min_update in fp32 on the GPU and
    # fp64 in the oracle, so a level's iteration count may differ by one near
    # the threshold: at most one per level, 3 in total over these 3 levels;
    # positions then differ by less than min_update
    prev = synth.smooth_frame(752, 480, seed=13)
    nxt = synth.smooth_frame(752, 480, seed=13, dx=0.4, dy=1.9, gain=1.1, offset=-6.0)
    pts = grid(752, 480, 29, 40)
    got = run(det, [(prev, nxt)], [pts])[0]
    want = lk.track(prev, nxt, pts.astype(np.float64), levels=3)
    xy, gain, off, status, iters, res = vio.track_fields(got)
    assert np.array_equal(status, want[:, 4].astype(np.int32))
    tr = want[:, 4] == lk.TRACKED
    assert np.abs(xy[tr] - want[tr, :2]).max() < 0.02
    assert np.abs(iters - want[:, 5]).max() <= 3
    assert (np.abs(iters - want[:, 5]) == 0).mean() > 0.9


def test_features_from_the_detector(det):
    """Detect on one frame, track to the next: the frontend loop."""
    prev = synth.smooth_frame(752, 480, seed=14)
    nxt = synth.smooth_frame(752, 480, seed=14, dx=2.5, dy=1.25)
    outs, counts = det.detect([torch.from_numpy(prev).cuda()], 5, 9, 32, 3)
    det.sync()
    cells = outs[0].cpu().numpy()
    pts = cells[cells[:, 2] >= 0][:, :2].astype(np.float32)
    pts = pts[(pts[:, 0] >= 24) & (pts[:, 0] < 752 - 24) & (pts[:, 1] >= 24) & (pts[:, 1] < 480 - 24)]
    assert len(pts) > 50
    params = dict(levels=3, max_iters=15, min_update=0.0, model=0)
    got = run(det, [(prev, nxt)], [pts], **params)[0]
    L, kw = oracle_params(params)
    want, mask = converged(prev, nxt, pts.astype(np.float64), L, kw)
    assert mask.mean() >= 0.9
    assert_close(got, want, mask, exact_iters=True)
    xy = vio.track_fields(got)[0]
    assert np.median(np.abs(xy - (pts + [2.5, 1.25]))) < 0.05


def test_many_pairs_of_mixed_sizes_in_one_call(det):
    sizes = [(640, 480), (752, 480), (1280, 720), (320, 240)]
    pairs, pts = [], []
    for i in range(12):
        w, h = sizes[i % 4]
        prev = synth.smooth_frame(w, h, seed=100 + i)
        nxt = synth.smooth_frame(w, h, seed=100 + i, dx=0.3 * i - 1.5, dy=1.1 - 0.2 * i, gain=1.0 + 0.01 * i)
        pairs.append((prev, nxt))
        # pair 5 has no features: the prefix over pairs must skip it
        pts.append(np.zeros((0, 2), np.float32) if i == 5 else grid(w, h, 53, 30))
    params = dict(levels=3, max_iters=10, min_update=0.0, model=3)
    got = run(det, pairs, pts, **params)
    L, kw = oracle_params(params)
    for (prev, nxt), p, g in zip(pairs, pts, got):
        assert g.shape == (len(p), 8)
        if len(p) == 0:
            continue
        want, mask = converged(prev, nxt, p.astype(np.float64), L, kw)
        assert mask.mean() >= 0.9
        assert_close(g, want, mask, exact_iters=True)


def test_lost_tracks(det):
    img = synth.smooth_frame(320, 240, seed=15)
    flat = np.full((240, 320), 90, np.uint8)
    moved = synth.smooth_frame(320, 240, seed=15, dx=6.0)
    # template outside / inside; carried out of the next frame; tracked
    pts = np.array([[8.0, 100.0], [9.0, 100.0], [306.0, 120.0], [160.0, 120.0]], np.float32)
    params = dict(levels=1, max_iters=40, min_update=0.0, model=0)
    got = run(det, [(img, moved), (flat, flat)], [pts, pts], **params)
    L, kw = oracle_params(params)
    for (a, b), g in zip([(img, moved), (flat, flat)], got):
        want = lk.track(a, b, pts.astype(np.float64), levels=L, **kw)
        _, _, _, status, iters, _ = vio.track_fields(g)
        assert np.array_equal(status, want[:, 4].astype(np.int32))
        assert np.array_equal(iters, want[:, 5].astype(np.int32))
    assert vio.track_fields(got[0])[3].tolist() == [0, 1, 0, 1]
    assert vio.track_fields(got[1])[3].tolist() == [0, 0, 0, 0]


def test_unaligned_frames_match_aligned(det):
    prev = synth.smooth_frame(333, 241, seed=16)
    nxt = synth.smooth_frame(333, 241, seed=16, dx=1.0, dy=-0.5)
    pts = grid(333, 241, 31, 30)
    a = run(det, [(prev, nxt)], [pts], levels=3)[0]
    # pitch 345 and an odd base address force the copy into a context slot
    buf_p = torch.zeros(241 * 345 + 64, dtype=torch.uint8, device="cuda")
    buf_n = torch.zeros(241 * 345 + 64, dtype=torch.uint8, device="cuda")
    vp = buf_p[3:3 + 241 * 345].view(241, 345)[:, :333]
    vn = buf_n[3:3 + 241 * 345].view(241, 345)[:, :333]
    vp.copy_(torch.from_numpy(prev).cuda())
    vn.copy_(torch.from_numpy(nxt).cuda())
    q = torch.from_numpy(pts).cuda()
    b = det.track([vp], [vn], [q], dict(levels=3))[0]
    det.sync()
    assert np.array_equal(a, b.cpu().numpy())


def test_invalid_arguments(det):
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    q = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    for bad in (dict(levels=0), dict(levels=6), dict(patch_fine=12), dict(patch_coarse=4), dict(max_iters=0),
                dict(max_iters=101), dict(min_update=-1.0), dict(min_update=float("nan")), dict(model=4),
                dict(levels=5)):  # 64 >> 4 = 4 < 7: the smallest level is too small
        with pytest.raises(vio.VioError):
            det.track([img], [img], [q], bad)


def test_track_cells_from_the_detector(det):
    """The frontend loop without a copy of the features: the records of a
    detection of the previous frame are tracked as they are; every non-empty
    cell's track equals the oracle's from that cell's position, every empty
    cell gives an empty result."""
    prev = synth.smooth_frame(752, 480, seed=21)
    nxt = synth.smooth_frame(752, 480, seed=21, dx=-1.75, dy=2.5, gain=1.05, offset=-4.0)
    # a flat 5 x 5-cell block: the cells well inside it hold no corner on any level
    prev[160:320, 320:480] = 128
    nxt[160:320, 320:480] = 128
    gp, gn = torch.from_numpy(prev).cuda(), torch.from_numpy(nxt).cuda()
    outs, _ = det.detect([gp], 5, 9, 32, 3)
    params = dict(levels=3, max_iters=12, min_update=0.0, model=3)
    res = det.track_cells([gp], [gn], outs, params)[0]
    det.sync()
    cells = outs[0].cpu().numpy()
    got = res.cpu().numpy()
    xy, gain, off, status, iters, resid = vio.track_fields(got)
    empty = cells[:, 2] < 0
    assert empty.any() and (~empty).sum() > 50
    assert (status[empty] == 0).all() and (iters[empty] == 0).all() and (xy[empty] == -1).all()
    pts = cells[~empty][:, :2].astype(np.float64)
    L, kw = oracle_params(params)
    want, mask = converged(prev, nxt, pts, L, kw)
    assert mask.mean() >= 0.9
    assert_close(got[~empty], want, mask, exact_iters=True)
