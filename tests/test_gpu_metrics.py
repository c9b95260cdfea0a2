"""GPU accuracy measures (dc_metrics) against the oracle's: completed
synthetic frames scored against the scenes' ray-cast ground truth (the
KITTI measures of Section V, Tables 1-3)."""
import numpy as np
import pytest

import oracle
from paper_1802_00036_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00036_gb300 import build, dc
    build.build()
    c = dc.Context(0)
    yield c
    c.close()


def test_metrics_match_oracle(ctx):
    from paper_1802_00036_gb300 import dc
    spec = synth.FrameSpec(176, 608, 32, 0.05, 2.0, 80.0)
    seeds = [synth.frame_seed(3, i) for i in range(4)]
    sparse = np.stack([synth.make_frame(spec, s) for s in seeds])
    gt = np.stack([synth.ground_truth(spec, s) for s in seeds])
    x = torch.from_numpy(sparse).cuda()
    y = torch.empty_like(x)
    ctx.complete(x, y)
    g = torch.from_numpy(gt).cuda()
    got = dc.dc_metrics(ctx.h, y.data_ptr(), g.data_ptr(), 4, spec.H, spec.W)
    pred = y.cpu().numpy()
    for i in range(4):
        want = oracle.metrics(pred[i], gt[i])
        assert got[i][4] == want["valid"]
        for j, k in enumerate(("rmse_mm", "mae_mm", "irmse_per_km", "imae_per_km")):
            assert got[i][j] == pytest.approx(want[k], rel=1e-5, abs=1e-6), (i, k)
    # a completed map is far closer to the truth than the sparse input
    assert got[0][0] < oracle.metrics(sparse[0], gt[0])["rmse_mm"]


def test_metrics_empty_truth_and_ragged_size(ctx):
    from paper_1802_00036_gb300 import dc
    H, W = 37, 71
    gt = np.zeros((2, H, W), np.float32)
    gt[1, 5:9, 7:40] = 15.0
    pred = np.full((2, H, W), 14.0, np.float32)
    dp, dg = torch.from_numpy(pred).cuda(), torch.from_numpy(gt).cuda()   # keep both alive
    got = dc.dc_metrics(ctx.h, dp.data_ptr(), dg.data_ptr(), 2, H, W)
    assert got[0] == (0.0, 0.0, 0.0, 0.0, 0.0)
    assert got[1][4] == 4 * 33 and got[1][0] == pytest.approx(1000.0) and got[1][1] == pytest.approx(1000.0)


def test_projection_matches_oracle_bit_exact(ctx):
    from paper_1802_00036_gb300 import dc
    for spec, seed in ((synth.ONE_FRAME, 11), (synth.FrameSpec(375, 1242, 64, 0.06, 1.0, 90.0), 12)):
        pts = synth.point_cloud(spec, seed, extra=50000)
        P = synth.camera_matrix(spec)
        want = oracle.project(pts, P, spec.H, spec.W, spec.d_min, spec.d_max)
        dpts = torch.from_numpy(pts).cuda()
        out = torch.full((spec.H, spec.W + 8), -1.0, device="cuda")      # pitched output
        dc.dc_project(ctx.h, dpts.data_ptr(), len(pts), P.ravel(), spec.H, spec.W, spec.d_min, spec.d_max,
                      out.data_ptr(), spec.W + 8)
        torch.cuda.synchronize()
        got = out[:, :spec.W].cpu().numpy()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        assert np.all(out[:, spec.W:].cpu().numpy() == -1.0)          # padding untouched
        # and the projected map feeds the chain like the sparse frame it came from
        np.testing.assert_array_equal(got[synth.make_frame(spec, seed) > 0] > 0, True)


def test_projection_of_no_points_is_empty(ctx):
    from paper_1802_00036_gb300 import dc
    out = torch.full((9, 13), 5.0, device="cuda")
    dc.dc_project(ctx.h, 0, 0, np.eye(3, 4).ravel(), 9, 13, 0.1, 100.0, out.data_ptr())
    torch.cuda.synchronize()
    assert torch.all(out == 0)
