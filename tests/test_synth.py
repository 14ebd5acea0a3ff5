"""The seeded frame generator gives the recorded bytes (tests/golden/frame_sha256.txt,
written by tests/golden/make_frame_hashes.py): every workload's inputs are the
same on every host."""
import os

import pytest

from paper_2003_13493_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "frame_sha256.txt")


def cases():
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w, h, seed, ns, digest = line.split()
                yield int(w), int(h), int(seed), int(ns), digest


def check_all():
    for w, h, seed, ns, digest in cases():
        assert synth.frame_sha256(synth.make_frame(w, h, seed=seed, n_shapes=ns)) == digest, (w, h, seed)


def test_frames_match_recorded_hashes():
    check_all()


@pytest.mark.gpu
def test_frames_match_recorded_hashes_on_the_gpu_host():
    # the GPU parity tests generate their inputs on the GPU's host
    check_all()


def test_mixed_batch_layout():
    frames = synth.mixed_batch(first_seed=2, per_size=16)
    assert len(frames) == 64
    sizes = [f.shape[::-1] for f in frames]
    for i, (w, h) in enumerate(synth.MIXED_SIZES):
        assert sizes[16 * i:16 * i + 16] == [(w, h)] * 16
    assert synth.frame_sha256(frames[0]) == synth.frame_sha256(synth.make_frame(640, 480, seed=2))
