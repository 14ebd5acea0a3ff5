"""The allocation-free entry point (vio_detect_noalloc), called through the
C ABI, must give exactly what vio_detect gives, call after call.

It serves callers that cannot allocate device memory when they detect (a
pool that accounts for every byte, a real-time loop that cannot afford
cudaMalloc's synchronisation, a plug-in whose host owns all allocations);
its working memory is one fixed array inside the library.  This file is
collected last so that a run stopping at its first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

from paper_2003_13493_gb300 import synth, vio

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc(lib, frame, thresh, arc, cell, levels, score=0, with_count=True):
    h, w = frame.shape
    out = torch.full((vio.num_cells(w, h, cell), 4), 7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    st = lib.vio_detect_noalloc(ctypes.c_void_p(frame.data_ptr()), vio.Dims(w, h, frame.stride(0)), thresh, arc,
                                cell, levels, score, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(cnt.data_ptr() if with_count else None),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out, cnt


def _reference(frame, thresh, arc, cell, levels, score=0):
    det = vio.Detector(max_frames=2, score=score)
    outs, counts = det.detect([frame], thresh, arc, cell, levels)
    det.sync()
    r = outs[0].cpu().numpy(), int(counts[0])
    det.close()
    return r


CASES = [((752, 480, 1), 20, 9, 32, 3, 0), ((1920, 1080, 60), 15, 9, 32, 3, 0),
         ((3840, 2160, 100), 10, 12, 64, 4, 0), ((640, 480, 3), 15, 9, 32, 3, 2)]


def test_noalloc_matches_vio_detect_on_consecutive_calls():
    lib = vio.load()
    for (w, h, seed), thresh, arc, cell, levels, score in CASES:
        frames = [torch.from_numpy(synth.make_frame(w, h, seed=seed + j,
                                                    n_shapes=400 if w > 2000 else 40)).cuda() for j in range(2)]
        # two calls in a row on the same stream share the library's array
        results = [_noalloc(lib, f, thresh, arc, cell, levels, score) for f in frames]
        torch.cuda.synchronize()
        for f, (st, out, cnt) in zip(frames, results):
            assert st == 0, (w, h, st)
            ref, n = _reference(f, thresh, arc, cell, levels, score)
            assert np.array_equal(out.cpu().numpy(), ref), (w, h)
            assert int(cnt[0]) == n


def _strided(w, h, seed, pad):
    """A frame seen through a row-strided view: pitch w + pad bytes."""
    full = torch.zeros((h, w + pad), dtype=torch.uint8, device="cuda")
    full[:, :w] = torch.from_numpy(synth.make_frame(w, h, seed=seed)).cuda()
    return full[:, :w]


# branches the cases above leave out: one level (no pyramid launch, no level
# maps), the SAD-A score, a pitch larger than the width, and no count output
BRANCH_CASES = [
    dict(w=752, h=480, seed=0, thresh=10, arc=9, cell=32, levels=1, score=0, pad=0, with_count=True),
    dict(w=752, h=480, seed=5, thresh=20, arc=10, cell=32, levels=3, score=1, pad=0, with_count=True),
    dict(w=752, h=480, seed=6, thresh=15, arc=9, cell=64, levels=3, score=0, pad=64, with_count=True),
    dict(w=640, h=480, seed=7, thresh=15, arc=9, cell=32, levels=2, score=0, pad=0, with_count=False),
]


@pytest.mark.parametrize("case", BRANCH_CASES, ids=["one-level", "sad-a", "strided", "no-count"])
def test_noalloc_branches_match_vio_detect(case):
    lib = vio.load()
    c = dict(case)
    frames = [_strided(c["w"], c["h"], c["seed"] + j, c["pad"]) for j in range(2)]
    assert frames[0].stride(0) == c["w"] + c["pad"]
    results = [_noalloc(lib, f, c["thresh"], c["arc"], c["cell"], c["levels"], c["score"], c["with_count"])
               for f in frames]
    torch.cuda.synchronize()
    for f, (st, out, cnt) in zip(frames, results):
        assert st == 0, (c, st)
        ref, n = _reference(f, c["thresh"], c["arc"], c["cell"], c["levels"], c["score"])
        assert np.array_equal(out.cpu().numpy(), ref), c
        if c["with_count"]:
            assert int(cnt[0]) == n
        else:
            assert int(cnt[0]) == -5  # no count pointer: nothing written there


def test_noalloc_rejects_frames_beyond_the_array():
    lib = vio.load()
    big = torch.zeros((4000, 4000), dtype=torch.uint8, device="cuda")
    st, out, cnt = _noalloc(lib, big, 10, 9, 32, 2)
    torch.cuda.synchronize()
    assert st == 1  # VIO_ERR_INVALID_ARG: 2048 x 2000 level-1 pixels exceed the array
    assert (out == 7).all() and int(cnt[0]) == -5  # nothing was enqueued
