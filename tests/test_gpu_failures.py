"""Failure handling, tested without any failure on the GPU: the context is
put into the state a failure would leave (dc_inject_fault), or a serving
client misbehaves on the host.  Each time, the error is reported where
include/dc.h says, exactly once, and the context keeps producing the
oracle's results afterwards."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1802_00036_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_BLUR_M = 1e-4
SPEC = synth.FrameSpec(96, 200, 16, 0.05, 2.0, 80.0)


@pytest.fixture(scope="module")
def dc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00036_gb300 import build, dc as dcmod
    build.build()
    return dcmod


def _run_and_check(dc, ctx):
    f = synth.make_frame(SPEC, 31)
    got = ctx.complete(torch.from_numpy(f).cuda()).cpu().numpy()
    assert np.abs(got.astype(np.float64) - oracle.complete(f)).max() <= TOL_BLUR_M


def test_a_wait_that_gave_up_is_reported_once(dc):
    ctx = dc.Context(0)
    try:
        _run_and_check(dc, ctx)
        dc.dc_inject_fault(ctx.h, dc.DC_FAULT_WAIT)
        assert dc.dc_last_async_error(ctx.h) == dc.DC_ERR_TIMEOUT
        assert dc.dc_last_async_error(ctx.h) == dc.DC_OK
        _run_and_check(dc, ctx)
        assert dc.dc_last_async_error(ctx.h) == dc.DC_OK
    finally:
        ctx.close()


def test_a_refused_launch_fails_its_call_and_is_reported(dc):
    ctx = dc.Context(0)
    try:
        f = torch.from_numpy(synth.make_frame(SPEC, 32)).cuda()
        out = torch.full_like(f, -3.0)
        dc.dc_inject_fault(ctx.h, dc.DC_FAULT_LAUNCH)
        with pytest.raises(dc.DcError) as e:
            dc.dc_complete_uniform(ctx.h, f.data_ptr(), out.data_ptr(), 1, SPEC.H, SPEC.W, dc.params())
        assert e.value.status == dc.DC_ERR_CUDA
        torch.cuda.synchronize()
        assert torch.all(out == -3.0)                     # nothing was queued
        assert dc.dc_last_async_error(ctx.h) == dc.DC_ERR_CUDA
        assert dc.dc_last_async_error(ctx.h) == dc.DC_OK
        _run_and_check(dc, ctx)
    finally:
        ctx.close()


def test_unknown_fault_is_refused(dc):
    ctx = dc.Context(0)
    try:
        with pytest.raises(dc.DcError) as e:
            dc.dc_inject_fault(ctx.h, 7)
        assert e.value.status == dc.DC_ERR_INVALID_ARG
    finally:
        ctx.close()


def test_a_stalled_sensor_does_not_hold_up_the_others(dc):
    # four client threads share a native server; the first submits a burst and
    # then stalls (never submits again, never polls).  The others keep
    # submitting and collecting: their results equal the frames run alone and
    # their latencies stay far below the stall; the stalled sensor's frames
    # are completed in its buffers all the same
    from paper_1802_00036_gb300.serve import NativeServer
    frames = [torch.from_numpy(synth.make_frame(SPEC, 600 + i)).pin_memory() for i in range(16)]
    outs = {}
    srv = NativeServer(max_hw=(SPEC.H, SPEC.W), budget_bytes=256 << 20, deadline_ms=1.0, max_batch=8, lanes=2)
    done = {}
    lock = threading.Lock()
    stop = threading.Event()

    def client(sensor, n_frames, polls):
        for k in range(n_frames):
            tag = sensor * 1000 + k
            f = frames[(sensor * 5 + k) % len(frames)]
            o = torch.full_like(f, -1.0).pin_memory()
            outs[tag] = (f, o)
            srv.submit(f.data_ptr(), o.data_ptr(), SPEC.H, SPEC.W, tag)
            time.sleep(0.002)
            if polls:
                with lock:
                    for t, ms in srv.poll():
                        done[t] = ms
        if polls:
            t_end = time.time() + 30
            while time.time() < t_end and not all(sensor * 1000 + k in done for k in range(n_frames)):
                with lock:
                    for t, ms in srv.poll():
                        done[t] = ms
                time.sleep(1e-3)

    stalled = threading.Thread(target=client, args=(0, 12, False))
    stalled.start()
    stalled.join()
    others = [threading.Thread(target=client, args=(s, 20, True)) for s in (1, 2, 3)]
    t0 = time.time()
    for t in others:
        t.start()
    for t in others:
        t.join()
    wall_ms = (time.time() - t0) * 1e3
    try:
        for s in (1, 2, 3):
            lat = [done[s * 1000 + k] for k in range(20)]
            assert len(lat) == 20 and max(lat) < 200.0 and max(lat) < wall_ms, (s, max(lat))
        # the stalled sensor's frames ran too: their tags wait in the done queue
        t_end = time.time() + 30
        while time.time() < t_end and not all(k in done for k in range(12)):
            for t, ms in srv.poll():
                done[t] = ms
            time.sleep(1e-3)
        assert all(k in done for k in range(12))
        st = srv.stats()
        assert st["submitted"] == 72 and st["done"] == 72
    finally:
        srv.close()
    ctx = dc.Context(0)
    try:
        for tag, (f, o) in outs.items():
            alone = ctx.complete(f.cuda()).cpu().numpy()
            assert np.array_equal(o.numpy().view(np.uint32), alone.view(np.uint32)), tag
    finally:
        ctx.close()


def test_a_client_that_leaves_with_frames_in_flight(dc):
    # frames submitted, then the server is destroyed at once without a poll:
    # destruction finishes every queued frame (their results land in the
    # callers' buffers) and returns
    from paper_1802_00036_gb300.serve import NativeServer
    frames = [torch.from_numpy(synth.make_frame(SPEC, 700 + i)).pin_memory() for i in range(10)]
    outs = [torch.full_like(f, -1.0).pin_memory() for f in frames]
    srv = NativeServer(max_hw=(SPEC.H, SPEC.W), budget_bytes=256 << 20, deadline_ms=5.0, max_batch=8, lanes=1)
    for i, (f, o) in enumerate(zip(frames, outs)):
        srv.submit(f.data_ptr(), o.data_ptr(), SPEC.H, SPEC.W, i)
    srv.close()
    ctx = dc.Context(0)
    try:
        for f, o in zip(frames, outs):
            alone = ctx.complete(f.cuda()).cpu().numpy()
            assert np.array_equal(o.numpy().view(np.uint32), alone.view(np.uint32))
    finally:
        ctx.close()
