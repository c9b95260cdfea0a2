"""The seeded inputs follow their recipe (the stand-in for KITTI depth
completion): whole-frame density at the target, returns only on the beams
over the lower two thirds, depths within the range and on KITTI's 1/256 m
grid, the batched workload's per-frame density drawn from its range, and a
frame determined by its seed alone."""
import numpy as np
import pytest

from paper_1802_00036_gb300 import synth


def _density(f):
    return float(np.count_nonzero(f)) / f.size


def test_one_frame_follows_the_recipe():
    spec = synth.ONE_FRAME
    f = synth.make_frame(spec, synth.frame_seed(0, 0))
    assert f.shape == (spec.H, spec.W) and f.dtype == np.float32
    assert 0.045 <= _density(f) <= 0.051
    rows = np.nonzero(f)[0]
    first_beam = spec.H / 3.0 + 0.5 * (2.0 * spec.H / 3.0) / spec.beams
    assert rows.min() >= np.floor(first_beam) - 1           # the upper third is empty
    assert rows.max() <= spec.H - 1
    v = f[f > 0]
    assert v.min() >= spec.d_min and v.max() <= spec.d_max
    assert np.array_equal(np.rint(v * 256.0) / 256.0, v)  # 16-bit fixed point, 1/256 m
    # beam pixels: at most three rows per beam after the wobble
    assert len(np.unique(rows)) <= 3 * spec.beams


def test_frames_depend_on_their_seed_only():
    a = synth.make_frame(synth.ONE_FRAME, 1234)
    b = synth.make_frame(synth.ONE_FRAME, 1234)
    c = synth.make_frame(synth.ONE_FRAME, 1235)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert not np.array_equal(a, c)


def test_batched_workload_densities_span_their_range():
    frames = synth.make_batch(12, synth.UNIFORM_375, config=2, density_range=(0.04, 0.06))
    d = np.array([_density(f) for f in frames])
    assert d.min() >= 0.037 and d.max() <= 0.061
    assert d.max() - d.min() > 0.005                       # drawn per frame, not one value
    v = frames[frames > 0]
    assert v.min() >= synth.UNIFORM_375.d_min and v.max() <= synth.UNIFORM_375.d_max


@pytest.mark.parametrize("spec", synth.MIX, ids=lambda s: f"{s.H}x{s.W}")
def test_mix_resolutions_hit_their_density(spec):
    f = synth.make_frame(spec, synth.frame_seed(3, 0))
    assert f.shape == (spec.H, spec.W)
    assert 0.88 * spec.density <= _density(f) <= 1.02 * spec.density
