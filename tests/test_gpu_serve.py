"""GPU tests of the serving loop: frames of several streams and sizes are
submitted one by one while earlier batches run; every result must equal the
oracle and a vio_detect of the same frame alone."""
import time

import numpy as np
import pytest

import oracle
from paper_2003_13493_gb300 import synth, vio

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PARAMS = dict(thresh=15, arc_len=9, cell_size=32, levels=3)


@pytest.fixture(scope="module")
def pool():
    frames = []
    for s, (w, h) in enumerate(synth.MIXED_SIZES):
        for j in range(3):
            frames.append((s, synth.make_frame(w, h, seed=700 + 10 * s + j)))
    return frames


def solo(frame):
    det = vio.Detector(max_frames=4)
    outs, counts = det.detect([torch.from_numpy(frame).cuda()], PARAMS["thresh"], PARAMS["arc_len"],
                              PARAMS["cell_size"], PARAMS["levels"])
    det.sync()
    r = outs[0].cpu().numpy(), int(counts[0])
    det.close()
    return r


def test_results_same_alone_and_in_the_mix(pool):
    det = vio.Detector(max_frames=64)
    det.serve_start(max_batch=6, lanes=3, **PARAMS)
    order = [(i * 7) % len(pool) for i in range(48)]  # interleaved streams and sizes
    tickets = []
    for i in order:
        sid, f = pool[i]
        tickets.append((det.submit(sid, f), i))
        if len(tickets) % 5 == 0:
            time.sleep(0.0005)  # let some batches start while others queue
    det.drain(60000)
    want = {}
    for t, i in tickets:
        _, f = pool[i]
        done, cells, cnt = det.poll(t, f.shape[1], f.shape[0])
        assert done
        if i not in want:
            ref, n = oracle.detect(f, PARAMS["thresh"], PARAMS["arc_len"], PARAMS["cell_size"], PARAMS["levels"])
            alone, n_alone = solo(f)
            assert np.array_equal(alone, ref) and n_alone == n
            want[i] = (ref, n)
        ref, n = want[i]
        assert np.array_equal(cells, ref), i
        assert cnt == n
    st = det.serve_stats()
    assert st["submitted"] == st["completed"] == len(tickets)
    assert st["batches"] >= 2 and st["p50_us"] <= st["p99_us"] <= st["max_us"]
    det.serve_stop()
    det.close()


def test_batches_form_and_lanes_overlap(pool):
    """A burst of frames submitted faster than one lane detects them: pending
    frames must be admitted as multi-frame batches into the free lanes, at
    least two lanes must hold batches at once, and some batches must overlap
    another lane's on the device timeline (CUDA events around each lane's
    work); every result still equals the oracle's."""
    keep, frames = [], []
    for sid, f in pool:
        buf = torch.empty(f.shape, dtype=torch.uint8).pin_memory()
        buf.numpy()[...] = f
        keep.append(buf)
        frames.append((sid, buf.numpy()))
    det = vio.Detector(max_frames=64)
    det.serve_start(max_batch=8, lanes=3, **PARAMS)
    order = [(i * 5) % len(frames) for i in range(120)]
    tickets = [(det.submit(*frames[i]), i) for i in order]
    det.drain(60000)
    st = det.serve_stats()
    want = {}
    for t, i in tickets:
        f = frames[i][1]
        done, cells, cnt = det.poll(t, f.shape[1], f.shape[0])
        assert done
        if i not in want:
            want[i] = oracle.detect(np.ascontiguousarray(f), PARAMS["thresh"], PARAMS["arc_len"],
                                    PARAMS["cell_size"], PARAMS["levels"])
        ref, n = want[i]
        assert np.array_equal(cells, ref) and cnt == n, i
    assert st["completed"] == len(tickets)
    assert st["max_batch_frames"] > 1 and st["mean_batch"] > 1.0, st
    assert st["max_lanes_in_flight"] >= 2, st
    assert st["overlapped_batches"] >= 1, st
    assert st["batches"] < len(tickets)
    det.serve_stop()
    det.close()


def test_queue_full_and_budget(pool):
    det = vio.Detector(max_frames=64)
    # a budget of ~2 large frames: frames are admitted as memory frees up
    det.serve_start(max_batch=16, lanes=2, queue_capacity=8, mem_budget_bytes=6 << 20, **PARAMS)
    accepted, busy = [], 0
    for k in range(40):
        sid, f = pool[k % len(pool)]
        s, t = det.submit_raw(sid, f.ctypes.data, vio.Dims(f.shape[1], f.shape[0], f.strides[0]))
        if s == 0:
            accepted.append((t, f))
        else:
            assert s == 5  # VIO_ERR_BUSY
            busy += 1
    det.drain(60000)
    assert busy > 0 and accepted
    for t, f in accepted:
        done, cells, cnt = det.poll(t, f.shape[1], f.shape[0])
        assert done
        ref, n = oracle.detect(f, PARAMS["thresh"], PARAMS["arc_len"], PARAMS["cell_size"], PARAMS["levels"])
        assert np.array_equal(cells, ref) and cnt == n
    assert det.serve_stats()["rejected"] == busy
    det.serve_stop()
    det.close()


def test_serving_errors():
    det = vio.Detector(max_frames=8)
    f = synth.make_frame(64, 64, seed=3)
    with pytest.raises(vio.VioError):
        det.submit(0, f)  # not serving
    det.serve_start(max_batch=4, lanes=1, **PARAMS)
    with pytest.raises(vio.VioError):
        det.serve_start(max_batch=4, lanes=1, **PARAMS)  # already serving
    with pytest.raises(vio.VioError):
        det.submit(0, np.zeros((20, 20), dtype=np.uint8))  # smallest level below 7x7
    with pytest.raises(vio.VioError):
        det.poll(12345, 64, 64)  # never issued
    t = det.submit(0, f)
    det.drain(10000)
    assert det.poll(t, 64, 64)[0]
    with pytest.raises(vio.VioError):
        det.poll(t, 64, 64)  # already taken
    det.serve_stop()
    det.close()


def test_lanes_inherit_score_and_nms_radius(pool):
    """Serving lanes score and suppress like the context that started them."""
    det = vio.Detector(max_frames=16, score=vio.SCORE_MT, nms_radius=2)
    det.serve_start(max_batch=4, lanes=2, **PARAMS)
    picks = pool[::3]
    tickets = [(det.submit(sid, f), f) for sid, f in picks]
    det.drain(60000)
    for t, f in tickets:
        done, cells, cnt = det.poll(t, f.shape[1], f.shape[0])
        assert done
        ref, n = oracle.detect(f, PARAMS["thresh"], PARAMS["arc_len"], PARAMS["cell_size"], PARAMS["levels"],
                               oracle.MT, nms_radius=2)
        assert np.array_equal(cells, ref) and cnt == n
    det.serve_stop()
    det.close()


def test_pinned_and_pageable_frames_in_one_mix(pool):
    """Pinned frames are read by the lanes' pyramid kernels through their
    device mapping, pageable or misaligned ones are copied; results must not
    depend on where a frame lives."""
    keep = []
    frames = []
    for k, (sid, f) in enumerate(pool):
        if k % 3 == 0:
            frames.append((sid, f))
            continue
        off = 0 if k % 3 == 1 else 1  # aligned / misaligned pinned
        buf = torch.empty(f.size + off + 64, dtype=torch.uint8).pin_memory()
        v = buf.numpy()[off:off + f.size].reshape(f.shape)
        v[...] = f
        keep.append(buf)
        frames.append((sid, v))
    det = vio.Detector(max_frames=32)
    det.serve_start(max_batch=5, lanes=3, **PARAMS)
    tickets = [(det.submit(sid, f), f) for sid, f in frames * 2]
    det.drain(60000)
    for t, f in tickets:
        done, cells, cnt = det.poll(t, f.shape[1], f.shape[0])
        assert done
        ref, n = oracle.detect(np.ascontiguousarray(f), PARAMS["thresh"], PARAMS["arc_len"], PARAMS["cell_size"],
                               PARAMS["levels"])
        assert np.array_equal(cells, ref) and cnt == n
    det.serve_stop()
    det.close()
