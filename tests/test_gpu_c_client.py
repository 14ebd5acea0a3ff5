"""The C ABI from plain C: tests/c_client/vio_client.c is compiled with the
host C compiler against include/vio.h, linked with the library and the CUDA
runtime, and run; its detections must equal the oracle's on the same frame
and its tracks must follow the frame's known shift."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2003_13493_gb300 import build, vio

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W, H = 640, 480


def frame():
    """The client's test frame (same formula as vio_client.c)."""
    y, x = np.mgrid[0:H, 0:W]
    v = 40 + (x + 2 * y) % 90
    sq = ((x // 24 + y // 24) % 3 == 0) & (x % 24 > 5) & (y % 24 > 7)
    v = np.where(sq, 200 + (x * 7 + y * 3) % 50, v)
    return np.ascontiguousarray(v.astype(np.uint8))


def test_c_client():
    lib = vio.load()
    assert lib is not None
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    out_dir = os.path.join(ROOT, "paper_2003_13493_gb300", "_build")
    exe = os.path.join(out_dir, "vio_client")
    cc = shutil.which("gcc") or shutil.which("cc")
    assert cc, "a host C compiler is needed"
    subprocess.check_call([cc, "-O2", "-std=c99", os.path.join(ROOT, "tests", "c_client", "vio_client.c"),
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                           "-L", out_dir, "-lvio_gb300", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                           "-Wl,-rpath," + out_dir, "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.splitlines()
    count = int(lines[0].split()[1])
    cells = np.array([[int(t) for t in ln.split()[2:]] for ln in lines if ln.startswith("cell ")], np.int32)
    want, n = oracle.detect(frame(), 15, 9, 32, 3)
    assert np.array_equal(cells, want) and count == n
    tracks = [ln.split()[1:] for ln in lines if ln.startswith("track ")]
    assert tracks
    for x, y, tx, ty, st in tracks:
        # interior features follow the whole-pixel shift exactly (residual zero there)
        assert int(st) == 1
        assert abs(float(tx) - (float(x) + 3)) < 0.05 and abs(float(ty) - (float(y) + 2)) < 0.05
