"""CPU checks of the C ABI: the library builds, loads and exports every
function include/vio.h declares; pure host helpers behave; without a GPU the
context constructor fails with a status instead of crashing."""
import ctypes

import pytest

from paper_2003_13493_gb300 import vio


@pytest.fixture(scope="module")
def lib():
    return vio.load()


def test_exports_every_declared_function(lib):
    names = vio.header_functions()
    assert "vio_detect" in names and "vio_create" in names and "vio_destroy" in names
    for name in names:
        assert hasattr(lib, name), name


def test_num_cells(lib):
    assert vio.num_cells(752, 480, 32) == 24 * 15
    assert vio.num_cells(1920, 1080, 32) == 60 * 34
    assert vio.num_cells(3840, 2160, 64) == 60 * 34
    assert vio.num_cells(32, 32, 32) == 1
    assert vio.num_cells(33, 32, 32) == 2
    assert vio.num_cells(0, 10, 32) == 0
    assert vio.num_cells(10, 10, 0) == 0


def test_status_strings(lib):
    for s in range(8):
        assert lib.vio_status_str(s)
    assert lib.vio_status_str(99) == b"unknown status"


def test_config_default(lib):
    cfg = vio.Config()
    lib.vio_config_default(ctypes.byref(cfg))
    assert (cfg.device, cfg.max_frames, cfg.score, cfg.autotune, cfg.use_graphs) == (0, 64, 0, 0, 1)
    assert cfg.nms_radius == 1


def test_variants_listed(lib):
    vs = vio.variants()
    assert len(vs) >= 3
    for tw, th, r in vs:
        # a score region of tw + 8 = 128 pixels (one warp of 4-pixel words per
        # row) and th + 2r rows split over 8 warps in groups of 4; the TMA box
        # adds the 3-row circle halo above and below
        assert 1 <= r <= 4
        assert tw + 8 == 128 and (th + 2 * r) % 32 == 0 and th + 2 * r + 6 <= 256
    # every NMS radius of Table III has a variant, the 3x3 one first
    assert vs[0][2] == 1 and sorted({r for _, _, r in vs}) == [1, 2, 3, 4]
    assert vio.variant_ids(1)[0] == 0 and len(vio.variant_ids(1)) >= 3
    t = vio.Tuning()
    assert lib.vio_variant(len(vs), ctypes.byref(t)) == 1


def test_create_rejects_bad_config_and_null(lib):
    assert lib.vio_create(None, None) == 1
    cfg = vio.Config()
    lib.vio_config_default(ctypes.byref(cfg))
    cfg.max_frames = 0
    ctx = ctypes.c_void_p()
    assert lib.vio_create(ctypes.byref(ctx), ctypes.byref(cfg)) == 1
    assert not ctx
    for r in (0, 5, -1):
        lib.vio_config_default(ctypes.byref(cfg))
        cfg.nms_radius = r
        assert lib.vio_create(ctypes.byref(ctx), ctypes.byref(cfg)) == 1
        assert not ctx
    assert lib.vio_get_config(None, ctypes.byref(cfg)) == 1


def test_destroy_null_is_noop(lib):
    assert lib.vio_destroy(None) == 0


def test_track_defaults_and_null_context(lib):
    p = vio.TrackParams()
    lib.vio_track_params_default(ctypes.byref(p))
    assert (p.levels, p.patch_fine, p.patch_coarse, p.max_iters, p.model) == (3, 16, 8, 30, 3)
    assert abs(p.min_update - 0.01) < 1e-7
    assert lib.vio_track(None, None, None, None, 0, None, None, None, None, None) == 1


def test_host_batch_marshals_once_and_checks_buffers():
    """HostBatch (host logic only): dims and pointers are taken from the
    arrays once; wrong dtypes, layouts or output counts are refused."""
    import numpy as np

    frames = [np.zeros((480, 640), np.uint8), np.zeros((720, 1280), np.uint8)[:, :1000]]
    outs = [np.zeros((vio.num_cells(f.shape[1], f.shape[0], 32), 4), np.int32) for f in frames]
    counts = np.zeros(2, np.int32)
    b = vio.HostBatch(frames, outs, counts)
    assert b.n == 2
    assert [(d.w, d.h, d.pitch) for d in b.dims] == [(640, 480, 640), (1000, 720, 1280)]
    assert [b.fptr[i] for i in range(2)] == [f.ctypes.data for f in frames]
    assert [b.optr[i] for i in range(2)] == [o.ctypes.data for o in outs]
    assert b.cptr.value == counts.ctypes.data
    assert vio.HostBatch(frames, outs).cptr is None
    with pytest.raises(ValueError):
        vio.HostBatch([np.zeros((8, 8), np.int16)], outs[:1])
    with pytest.raises(ValueError):
        vio.HostBatch([np.zeros((8, 8, 2), np.uint8)[:, :, 0]], outs[:1])  # column stride 2
    with pytest.raises(ValueError):
        vio.HostBatch(frames, outs[:1])
