"""The checked build (-DVIO_CHECKED: every queue, score-tile and cell index
of the detect kernels is bounds-checked, a failed check is reported through
the status word and the access skipped) on the workloads and edge cases; run
in a child process that loads that build.  Its results must equal the
oracle and no check may fire."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
import oracle
from paper_2003_13493_gb300 import synth, vio
assert vio.lib_path().endswith("libvio_gb300.so")
def run(det, imgs, t, a, c, L, mode=0, r=1):
    fr = [torch.from_numpy(i).cuda() for i in imgs]
    outs, counts = det.detect(fr, t, a, c, L)
    det.sync()  # raises on any device-side status, the index checks included
    for i, im in enumerate(imgs):
        want, n = oracle.detect(im, t, a, c, L, mode, nms_radius=r)
        assert np.array_equal(outs[i].cpu().numpy(), want), (im.shape, t, a, c, L, mode, r)
        assert int(counts[i]) == n
mixed = synth.mixed_batch(first_seed=2, per_size=16)
for mode in (0, 1, 2):
    det = vio.Detector(max_frames=64, score=mode)
    run(det, mixed[::5], 15, 9, 32, 3, mode)
    det.close()
for r in (2, 4):
    det = vio.Detector(max_frames=16, nms_radius=r)
    run(det, mixed[::9], 15, 12, 64, 3, 0, r)
    det.close()
det = vio.Detector(max_frames=64)
for v in vio.variant_ids(1):
    det.set_variant(v)
    run(det, mixed[::7], 5, 9, 32, 3)
det.set_variant(None)
for (w, h, L) in [(7, 7, 1), (31, 17, 1), (257, 131, 3), (4000, 70, 3), (1920, 1080, 5)]:
    run(det, [synth.make_frame(w, h, seed=w + h)], 10, 9, 32, L)
fr = [torch.from_numpy(i).cuda() for i in mixed[::8]]
outs, counts = det.detect_sweep(fr, [(5, 12), (10, 9), (20, 9), (40, 16)], 32, 3)
det.sync()
for p, (t, a) in enumerate([(5, 12), (10, 9), (20, 9), (40, 16)]):
    for i, im in enumerate(mixed[::8]):
        want, n = oracle.detect(im, t, a, 32, 3)
        assert np.array_equal(outs[p][i].cpu().numpy(), want)
det.close()
print("checked build ok")
"""


def test_checked_build_runs_clean():
    from paper_2003_13493_gb300 import build

    path = build.build(checked=True)
    assert os.path.exists(path)
    env = dict(os.environ, VIO_CHECKED="1", PYTHONPATH=ROOT)
    child = CHILD.replace('endswith("libvio_gb300.so")', 'endswith("libvio_gb300_checked.so")')
    r = subprocess.run([sys.executable, "-c", child], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
