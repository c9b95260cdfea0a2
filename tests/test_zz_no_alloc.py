"""The allocation-free entry point, dc_complete_noalloc, against the regular
dc_complete_uniform on the same frames.

dc_complete_noalloc exists for callers that cannot allocate device memory
at run time (fixed memory plans, plug-ins handed their buffers by a host
framework); its scratch is one fixed array inside the library that every
call shares.  This file is named to be collected last, so a failure here
comes after every other test has run; it also passes on its own in a fresh
process, because the entry point sets itself up on its first call.
"""
import numpy as np
import pytest

from paper_1802_00036_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_BLUR_M = 1e-4   # the tolerance of the parity tests, metres, after the blur


@pytest.fixture(scope="module")
def dc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_00036_gb300 import build, dc as dcmod
    build.build()
    return dcmod


def _same(got, want, exact):
    if exact:
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    else:
        assert np.abs(got.astype(np.float64) - want).max() <= TOL_BLUR_M


@pytest.mark.parametrize("stop,exact", [("median", True), ("full", False)])
def test_noalloc_matches_regular_entry_point_twice(dc, stop, exact):
    spec = synth.FrameSpec(176, 608, 32, 0.05, 2.0, 80.0)
    ctx = dc.Context(0)
    try:
        p = dc.params(stop_after=stop)
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):                      # two calls in a row, new frames each time
            frames = synth.make_batch(3, spec, config=9, first=10 * call)
            x = torch.from_numpy(frames).cuda()
            y_ref = torch.full_like(x, -5.0)
            y_new = torch.full_like(x, -9.0)
            dc.dc_complete_uniform(ctx.h, x.data_ptr(), y_ref.data_ptr(), 3, spec.H, spec.W, p, stream)
            dc.dc_complete_noalloc(x.data_ptr(), y_new.data_ptr(), 3, spec.H, spec.W, p, stream)
            torch.cuda.synchronize()
            _same(y_new.cpu().numpy(), y_ref.cpu().numpy(), exact)
    finally:
        ctx.close()


def test_noalloc_refuses_sizes_beyond_its_array(dc):
    x = torch.zeros((1, 8, 8), device="cuda")
    y = torch.zeros_like(x)
    p = dc.params()
    with pytest.raises(dc.DcError) as e:        # 65 frames > DC_NOALLOC_MAX_FRAMES
        dc.dc_complete_noalloc(x.data_ptr(), y.data_ptr(), 65, 1, 1, p)
    assert e.value.status == 5
    big_in = torch.zeros((2048, 2048), device="cuda")
    big_out = torch.zeros_like(big_in)
    with pytest.raises(dc.DcError) as e:        # 2048 x 2048 > DC_NOALLOC_MAX_PIXELS
        dc.dc_complete_noalloc(big_in.data_ptr(), big_out.data_ptr(), 1, 2048, 2048, p)
    assert e.value.status == 5
