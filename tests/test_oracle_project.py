"""Pins of the oracle's LIDAR-to-image projection (Section V): points lifted
from a sparse map at their pixel centres project back onto it; the nearest
of several points in one pixel wins; points behind the camera, outside the
image or outside the depth range are dropped."""
import numpy as np

import oracle
from paper_1802_00036_gb300 import synth


def test_lifted_points_project_back_onto_their_map():
    spec = synth.FrameSpec(96, 160, 16, 0.08, 2.0, 80.0)
    frame = synth.make_frame(spec, 31)
    lifted = synth.point_cloud(spec, 31, extra=0)
    back = oracle.project(lifted, synth.camera_matrix(spec), spec.H, spec.W, spec.d_min, spec.d_max)
    np.testing.assert_array_equal(back, frame)
    # extra points can only add pixels or bring nearer depths
    full = oracle.project(synth.point_cloud(spec, 31, extra=3000), synth.camera_matrix(spec),
                          spec.H, spec.W, spec.d_min, spec.d_max)
    had = frame > 0
    assert np.all(full[had] <= frame[had]) and np.all(full[had] > 0)


def test_nearest_point_wins_and_filters():
    P = np.array([[10.0, 0, 5.0, 0], [0, 10.0, 5.0, 0], [0, 0, 1.0, 0]])
    pts = np.array([[0.0, 0.0, 4.0],      # pixel (5, 5), depth 4
                    [0.01, 0.01, 2.0],    # same pixel, nearer
                    [0.0, 0.0, -3.0],     # behind the camera
                    [100.0, 0.0, 1.0],    # outside the image
                    [0.2, 0.2, 200.0]],   # beyond d_max
                   np.float32)
    d = oracle.project(pts, P, 10, 10, 0.1, 100.0)
    assert d[5, 5] == np.float32(2.0) and np.count_nonzero(d) == 1
