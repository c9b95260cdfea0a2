"""Continuous-batching server: every frame's result is the same whether it
is processed alone or inside a served mix of sensors, sizes and batches
(the per-frame arithmetic does not depend on the batch)."""
import numpy as np
import pytest

from paper_1802_00036_gb300 import synth

torch = pytest.importorskip("torch")


def test_poisson_schedule_is_sorted_and_rate_plausible():
    from paper_1802_00036_gb300.serve import poisson_schedule
    t, s = poisson_schedule(200.0, 8, 2.0, seed=3)
    assert np.all(np.diff(t) >= 0) and set(np.unique(s)) <= set(range(8))
    assert abs(len(t) - 3200) < 4 * np.sqrt(3200)


@pytest.mark.gpu
def test_served_results_equal_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00036_gb300 import build, dc
    from paper_1802_00036_gb300.serve import Server
    build.build()
    specs = [synth.FrameSpec(352, 1216, 64, 0.05), synth.FrameSpec(512, 2048, 128, 0.08),
             synth.FrameSpec(256, 512, 32, 0.03)]
    frames = [synth.make_frame(specs[i % 3], 7000 + i) for i in range(24)]
    srv = Server(max_hw=(512, 2048), budget_bytes=1 << 30, deadline_ms=3.0, max_batch=8, lanes=2)
    try:
        futs = [srv.submit(f, sensor=i % 4) for i, f in enumerate(frames)]
        got = [f.result(timeout=60) for f in futs]
        st = srv.stats().summary()
    finally:
        srv.close()
    assert st["frames"] == 24 and st["batches"] >= 3
    ctx = dc.Context(0)
    try:
        for f, g in zip(frames, got):
            alone = ctx.complete(torch.from_numpy(f).cuda()).cpu().numpy()
            assert np.array_equal(alone.view(np.uint32), g.view(np.uint32))
    finally:
        ctx.close()
