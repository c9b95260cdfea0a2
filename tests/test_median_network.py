"""The 5x5 median network of stage B (step 7 of arXiv 1802.00036, Section
IV-7), checked on its description before it reaches the GPU:

* the committed median_net.cuh is exactly what gen_median.py emits;
* every output of the 2 x 8 block reads only its own 25 inputs and selects
  the 13th smallest on all 2^25 binary windows (0-1 principle);
* on random real values (with ties) it agrees with numpy's median.
"""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_00036_gb300", "csrc")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("gen_median", os.path.join(CSRC, "gen_median.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_committed_header_is_generated(gen):
    with open(os.path.join(CSRC, "median_net.cuh")) as fh:
        assert fh.read() == gen.HEADER + gen.emit(8)


def test_zero_one_principle_every_output(gen):
    assert gen.verify(8) == 16 * (1 << 25)


def _eval_real(gen, vals):
    net, x, outs = gen.build(8)
    order, ops = gen.prune_and_fuse(net, outs)
    v = {}
    for r in range(6):
        for j in range(12):
            v[x[r][j]] = vals[r][j]
    for i in order:
        k = ops[i][0]
        if k == "in":
            continue
        a = [v[j] for j in ops[i][1:]]
        v[i] = min(a) if k.startswith("min") else max(a)
    return {key: v[w] for key, w in outs.items()}


@pytest.mark.parametrize("seed", range(20))
def test_random_real_windows(gen, seed):
    rng = np.random.default_rng(seed)
    vals = rng.integers(0, 6 if seed % 2 else 1000, size=(6, 12)).astype(np.float32)
    got = _eval_real(gen, vals)
    for (row, o), m in got.items():
        assert m == np.median(vals[row:row + 5, o:o + 5])


def test_op_count_is_what_the_header_states(gen):
    n, per = gen.count(8)
    assert per < 60.0
    with open(os.path.join(CSRC, "median_net.cuh")) as fh:
        assert f": {n} min/max" in fh.read()
