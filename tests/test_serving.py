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
def test_native_server_results_equal_alone():
    # libdc's serving worker: frames of three sizes from four sensors, batched
    # by size and deadline on two lanes; every result equals the frame run alone
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00036_gb300 import build, dc
    from paper_1802_00036_gb300.serve import NativeServer
    build.build()
    specs = [synth.FrameSpec(352, 1216, 64, 0.05), synth.FrameSpec(512, 2048, 128, 0.08),
             synth.FrameSpec(256, 512, 32, 0.03)]
    frames = [torch.from_numpy(synth.make_frame(specs[i % 3], 8000 + i)).pin_memory() for i in range(30)]
    outs = [torch.full_like(f, -1.0).pin_memory() for f in frames]
    srv = NativeServer(max_hw=(512, 2048), budget_bytes=1 << 30, deadline_ms=3.0, max_batch=8, lanes=2)
    done = {}
    try:
        for i, (f, o) in enumerate(zip(frames, outs)):
            srv.submit(f.data_ptr(), o.data_ptr(), f.shape[0], f.shape[1], 100 + i)
        import time
        t_end = time.time() + 60
        while len(done) < len(frames) and time.time() < t_end:
            for tag, ms in srv.poll():
                done[tag] = ms
            time.sleep(1e-3)
        st = srv.stats()
        with pytest.raises(dc.DcError):
            srv.submit(frames[0].data_ptr(), outs[0].data_ptr(), 600, 100, 1)  # beyond max_hw
    finally:
        srv.close()
    assert sorted(done) == list(range(100, 130)) and all(ms > 0 for ms in done.values())
    assert st["done"] == 30 and st["submitted"] == 30 and st["batches"] >= 4 and st["slots"] > 0
    ctx = dc.Context(0)
    try:
        for f, o in zip(frames, outs):
            alone = ctx.complete(f.cuda()).cpu().numpy()
            assert np.array_equal(o.numpy().view(np.uint32), alone.view(np.uint32))
    finally:
        ctx.close()


@pytest.mark.gpu
def test_native_server_deadline_closes_a_small_batch():
    # one frame, batches of up to 64: it runs when its 1 ms deadline passes
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import time
    from paper_1802_00036_gb300 import build, dc
    from paper_1802_00036_gb300.serve import NativeServer
    build.build()
    f = torch.from_numpy(synth.make_frame(synth.FrameSpec(256, 512, 32, 0.05), 9001)).pin_memory()
    o = torch.empty_like(f).pin_memory()
    srv = NativeServer(max_hw=(256, 512), budget_bytes=512 << 20, deadline_ms=1.0, max_batch=64, lanes=1)
    try:
        srv.submit(f.data_ptr(), o.data_ptr(), 256, 512, 7)
        got = []
        t_end = time.time() + 30
        while not got and time.time() < t_end:
            got = srv.poll()
            time.sleep(1e-3)
        assert [t for t, _ in got] == [7] and got[0][1] >= 1.0
        assert srv.stats()["batches"] == 1
    finally:
        srv.close()
    with pytest.raises(dc.DcError):
        dc.dc_server_create(0, 0, 512, 512 << 20, 1000, 64, 1, dc.params())
