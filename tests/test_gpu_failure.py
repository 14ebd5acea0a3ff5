"""Failure detection on the GPU without a fault: every device-side wait is
bounded; a wait that runs out records a status word that the host reads, and
the context stays usable afterwards."""
import time

import numpy as np
import pytest

import oracle
from paper_2003_13493_gb300 import synth, vio

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_reports_timeout_and_context_survives():
    det = vio.Detector(max_frames=4)
    t0 = time.perf_counter()
    st = det.lib.vio_selftest_timeout(det.ctx, 50000)  # 50 ms
    dt = time.perf_counter() - t0
    assert st == 4, vio.STATUS.get(st, st)  # VIO_ERR_TIMEOUT
    assert dt >= 0.05
    assert det.lib.vio_selftest_timeout(det.ctx, 0) == 1  # out of range
    # the status word was cleared and the context still detects correctly
    img = synth.make_frame(640, 480, seed=77)
    outs, counts = det.detect([torch.from_numpy(img).cuda()], 15, 9, 32, 3)
    det.sync()
    want, n = oracle.detect(img, 15, 9, 32, 3)
    assert np.array_equal(outs[0].cpu().numpy(), want) and int(counts[0]) == n
    det.close()
