"""Writes the golden fixtures of the oracle (run from the repo root:
``python tests/golden/make_golden.py``).

Only the oracle and the seeded input generator are called; no value here
comes from the GPU library.  The fixtures pin the oracle against itself
across machines and compilers: chain_small.txt holds a hand-built 14 x 18
map with two scan lines (Section IV's input: sparse rows, 0 = empty) and
the oracle's maps after steps 4, 5, 6, 7 (median), the blur and step 8,
as exact float hex; digests.txt holds SHA-256 digests of the seeded
352 x 1216 frame and of its oracle maps after step 4 and the median.
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1802_00036_gb300 import synth  # noqa: E402


def small_map():
    d = np.zeros((14, 18), np.float32)
    # two scan lines with gaps, a near object on the right, a far one left
    d[6, ::2] = np.linspace(12.0, 14.0, 9, dtype=np.float32)
    d[10, 1::3] = np.float32(9.5)
    d[6, 13:16] = np.float32(4.25)
    d[11, 2] = np.float32(31.0)
    d[6, 4] = 0.0
    return d


def write_small(path):
    d = small_map()
    with open(path, "w") as fh:
        fh.write("# arXiv 1802.00036 Section IV steps 1-8 on a hand-built 14x18 map;\n")
        fh.write("# written by tests/golden/make_golden.py from the oracle, float hex\n")
        blocks = [("input", d)]
        for st in ("fill7", "extend", "fill_large", "median", "blur", "full"):
            blocks.append((f"{st}:oracle", oracle.complete(d, stop_after=st)))
        for name, m in blocks:
            fh.write(f"@{name}\n")
            for row in m:
                fh.write(" ".join(float(x).hex() for x in row) + "\n")


def write_digests(path):
    d = synth.make_frame(synth.ONE_FRAME, synth.frame_seed(0, 0))
    with open(path, "w") as fh:
        fh.write("# SHA-256 of the seeded 352x1216 frame (config 0, frame 0) and of the\n")
        fh.write("# oracle's maps after step 4 and after the step-7 median; written by\n")
        fh.write("# tests/golden/make_golden.py\n")
        fh.write(f"input {hashlib.sha256(d.tobytes()).hexdigest()}\n")
        for st in ("fill7", "median"):
            h = hashlib.sha256(oracle.complete(d, stop_after=st).tobytes()).hexdigest()
            fh.write(f"{st} {h}\n")


if __name__ == "__main__":
    write_small(os.path.join(HERE, "chain_small.txt"))
    write_digests(os.path.join(HERE, "digests.txt"))
