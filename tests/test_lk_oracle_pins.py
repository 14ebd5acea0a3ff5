"""Pins of the tracker oracle (Section II-E, Eqs. 2-6) against what the
mathematics fixes: exact whole-pixel and sub-pixel motion with known ground
truth, a known affine intensity change, the model subsets of Table VI, the
photometric error being at a local minimum where the tracker stops, and the
degenerate cases (no motion, flat patch, patch leaving the image)."""
import numpy as np
import pytest

from oracle import lk_oracle as lk
from paper_2003_13493_gb300 import synth

FULL = lk.GAIN | lk.OFFSET
W, H = 320, 240


def grid_points(step=40, margin=40):
    ys, xs = np.mgrid[margin:H - margin + 1:step, margin:W - margin + 1:step]
    return np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.float64)


def test_identical_frames_do_not_move():
    img = synth.smooth_frame(W, H, seed=1)
    pts = grid_points()
    out = lk.track(img, img, pts, levels=3, model=FULL)
    assert (out[:, 4] == lk.TRACKED).all()
    # the residual is exactly zero, so the first update of every level is zero
    assert np.array_equal(out[:, :2], pts)
    assert (out[:, 2] == 0).all() and (out[:, 3] == 0).all()
    assert (out[:, 5] == 3).all() and (out[:, 6] == 0).all()


@pytest.mark.parametrize("dx,dy", [(3, -2), (-1, 4), (6, 5), (0, -7)])
def test_whole_pixel_shift_recovered(dx, dy):
    # bilinear samples at integer offsets are the pixels themselves, so the
    # photometric error is exactly zero at the true shift
    img = synth.smooth_frame(W, H, seed=2)
    nxt = synth.shift_frame(img, dx, dy)
    pts = grid_points()
    out = lk.track(img, nxt, pts, levels=3, model=0, max_iters=40, min_update=0.0)
    assert (out[:, 4] == lk.TRACKED).all()
    err = np.abs(out[:, :2] - (pts + [dx, dy]))
    assert err.max() < 1e-6, err.max()


@pytest.mark.parametrize("dx,dy", [(1.37, -0.62), (-2.25, 3.8), (0.5, 0.5)])
def test_subpixel_shift_recovered(dx, dy):
    prev = synth.smooth_frame(W, H, seed=3)
    nxt = synth.smooth_frame(W, H, seed=3, dx=dx, dy=dy)
    pts = grid_points()
    out = lk.track(prev, nxt, pts, levels=3, model=0, max_iters=30, min_update=1e-4)
    assert (out[:, 4] == lk.TRACKED).all()
    err = np.abs(out[:, :2] - (pts + [dx, dy]))
    # 8-bit rounding of both frames and the bilinear model error of the
    # smooth scene leave a few hundredths of a pixel
    assert err.max() < 0.05, err.max()
    assert np.median(err) < 0.02


def test_gain_and_offset_recovered():
    prev = synth.smooth_frame(W, H, seed=4)
    nxt = synth.smooth_frame(W, H, seed=4, dx=0.8, dy=-1.3, gain=0.85, offset=10.0)
    assert 0 < nxt.min() and nxt.max() < 255  # no clipping: the intensity model holds exactly
    pts = grid_points()
    out = lk.track(prev, nxt, pts, levels=3, model=FULL, max_iters=30, min_update=1e-4)
    assert (out[:, 4] == lk.TRACKED).all()
    # the bilinear model error of the moving scene, shared with the pure
    # translation cases, grows a little when alpha and beta absorb part of it
    assert np.abs(out[:, 0] - (pts[:, 0] + 0.8)).max() < 0.1
    assert np.abs(out[:, 1] - (pts[:, 1] - 1.3)).max() < 0.1
    assert np.abs(out[:, 2] + 0.15).max() < 0.01
    assert np.abs(out[:, 3] - 10.0).max() < 1.5
    # without the appearance terms the same pair is tracked worse
    out0 = lk.track(prev, nxt, pts, levels=3, model=0, max_iters=30, min_update=1e-4)
    assert np.median(out0[:, 6]) > 4 * np.median(out[:, 6])


@pytest.mark.parametrize("model,zero", [(0, (2, 3)), (lk.GAIN, (3,)), (lk.OFFSET, (2,))])
def test_model_subsets_leave_other_parameters_zero(model, zero):
    prev = synth.smooth_frame(W, H, seed=5)
    nxt = synth.smooth_frame(W, H, seed=5, dx=1.0, dy=0.5, gain=1.1, offset=5.0)
    out = lk.track(prev, nxt, grid_points(), levels=2, model=model)
    for c in zero:
        assert (out[:, c] == 0).all()
    for c in {2, 3} - set(zero):
        assert (out[:, c] != 0).any()


def ssd(nxt, prev, x, y, t, P=16):
    """Photometric error of a translation on level 0, evaluated directly."""
    off = np.arange(P) - (P - 1) / 2.0
    gx, gy = np.meshgrid(x + off, y + off)
    a, b = np.asarray(prev, np.float64), np.asarray(nxt, np.float64)

    def sample(img, u, v):
        u0, v0 = np.floor(u).astype(int), np.floor(v).astype(int)
        fu, fv = u - u0, v - v0
        return ((1 - fu) * (1 - fv) * img[v0, u0] + fu * (1 - fv) * img[v0, u0 + 1]
                + (1 - fu) * fv * img[v0 + 1, u0] + fu * fv * img[v0 + 1, u0 + 1])

    return float(np.sum((sample(b, gx + t[0], gy + t[1]) - sample(a, gx, gy)) ** 2))


def test_solution_is_near_the_photometric_error_minimum():
    # the inverse compositional fixed point weighs the residual with the
    # template gradient, the least-squares minimum with the image gradient;
    # they coincide when the residual vanishes (the whole-pixel case) and stay
    # within the interpolation error of the scene otherwise
    prev = synth.smooth_frame(W, H, seed=6)
    nxt = synth.smooth_frame(W, H, seed=6, dx=-1.7, dy=2.4)
    pts = grid_points()[::3]
    out = lk.track(prev, nxt, pts, levels=3, model=0, max_iters=50, min_update=1e-6)
    steps = np.linspace(-0.2, 0.2, 41)
    for (x, y), row in zip(pts, out):
        t = row[:2] - (x, y)
        costs = np.array([[ssd(nxt, prev, x, y, t + (u, v)) for u in steps] for v in steps])
        j, i = np.unravel_index(np.argmin(costs), costs.shape)
        assert np.hypot(steps[i], steps[j]) <= 0.12, (x, y, steps[i], steps[j])
        assert abs(t[0] + 1.7) < 0.1 and abs(t[1] - 2.4) < 0.1


def test_pyramid_extends_the_capture_range():
    prev = synth.smooth_frame(W, H, seed=7)
    nxt = synth.shift_frame(prev, 11, -9, fill=128)
    pts = grid_points(step=40, margin=60)

    def recovered(levels):
        o = lk.track(prev, nxt, pts, levels=levels, model=0, max_iters=40, min_update=1e-3)
        return ((o[:, 4] == lk.TRACKED) & (np.abs(o[:, :2] - (pts + [11, -9])).max(axis=1) < 0.01)).mean()

    # a 14-pixel motion: 1.75 pixels on level 3, far outside a 16 x 16
    # patch's basin on level 0 for the finer scene components
    deep, flat = recovered(4), recovered(1)
    assert deep == 1.0 and flat <= 0.7, (deep, flat)


def test_patch_leaving_the_image_is_lost():
    img = synth.smooth_frame(W, H, seed=8)
    # the 18 x 18 template grid of a 16 x 16 patch needs 8.5 pixels each side
    pts = np.array([[8.0, 100.0], [9.0, 100.0], [100.0, H - 10.0], [100.0, H - 11.0]])
    out = lk.track(img, img, pts, levels=1, model=0)
    assert out[:, 4].tolist() == [lk.LOST, lk.TRACKED, lk.LOST, lk.TRACKED]
    # motion that carries the patch out of the next frame
    nxt = synth.shift_frame(img, 12, 0)
    out = lk.track(img, nxt, np.array([[W - 14.0, 100.0]]), levels=1, model=0, max_iters=40)
    assert out[0, 4] == lk.LOST


def test_flat_patch_is_lost():
    img = np.full((H, W), 77, np.uint8)
    out = lk.track(img, img, grid_points(), levels=2, model=FULL)
    assert (out[:, 4] == lk.LOST).all() and (out[:, 5] == 0).all()
