"""Writes frame_sha256.txt: the SHA-256 of the seeded synthetic frames every
workload uses, so that a host whose generator produced other bytes is caught
(the generator is integer-only and must give the same bytes everywhere)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2003_13493_gb300 import synth  # noqa: E402

CASES = [(752, 480, 0, 40), (752, 480, 1, 40)]
CASES += [(w, h, 2 + 16 * i, 40) for i, (w, h) in enumerate(synth.MIXED_SIZES)]
CASES += [(3840, 2160, 100, 400), (64, 64, 3, 40), (7, 7, 11, 40)]


def main() -> None:
    with open(os.path.join(HERE, "frame_sha256.txt"), "w") as f:
        f.write("# w h seed n_shapes sha256 (synth.make_frame)\n")
        for w, h, seed, ns in CASES:
            f.write(f"{w} {h} {seed} {ns} {synth.frame_sha256(synth.make_frame(w, h, seed=seed, n_shapes=ns))}\n")


if __name__ == "__main__":
    main()
