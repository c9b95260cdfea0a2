"""The allocation-free entry point, dc_complete_noalloc, against the regular
dc_complete_uniform on the same frames and against the CPU oracle.

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


def _oracle_case(dc, frames, exact_stop, **kw):
    """dc_complete_noalloc on `frames` against the oracle, frame by frame."""
    import oracle
    x = torch.from_numpy(frames).cuda()
    y = torch.full_like(x, -9.0)
    n, H, W = frames.shape
    p = dc.params(**kw)
    dc.dc_complete_noalloc(x.data_ptr(), y.data_ptr(), n, H, W, p, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    for i in range(n):
        _same(got[i], oracle.complete(frames[i], **kw), exact_stop)


@pytest.mark.parametrize("stop", ["invert", "dilate", "close", "fill7", "extend", "fill_large", "median",
                                  "blur", "full"])
def test_noalloc_every_stop_against_the_oracle(dc, stop):
    # stops before step 5 run stage A alone, writing the output directly
    frames = synth.make_batch(2, synth.FrameSpec(96, 200, 16, 0.05, 2.0, 80.0), config=9, first=50)
    _oracle_case(dc, frames, stop not in ("blur", "full"), stop_after=stop)


@pytest.mark.parametrize("kw", [dict(blur="bilateral"), dict(blur="none", median=False),
                                dict(extend_top=False, large_fill_on=False), dict(extend_rows=8)])
def test_noalloc_variants_against_the_oracle(dc, kw):
    frames = synth.make_batch(2, synth.FrameSpec(120, 260, 32, 0.06, 1.0, 90.0), config=9, first=60)
    _oracle_case(dc, frames, False, **kw)


def test_noalloc_off_grid_depths_against_the_oracle(dc):
    # depths off the 1/256 m grid: the step-4 values go through the array's float part
    frames = np.stack([synth.random_sparse(90, 170, 0.08, 70 + i) for i in range(2)])
    _oracle_case(dc, frames, True, stop_after="median")
    _oracle_case(dc, frames, False)


def test_noalloc_at_its_limits(dc):
    # 64 frames of 32 x 1024: exactly DC_NOALLOC_MAX_PIXELS padded pixels and
    # DC_NOALLOC_MAX_FRAMES frames; sampled frames against the oracle
    import oracle
    spec = synth.FrameSpec(32, 1024, 8, 0.1, 2.0, 80.0)
    frames = synth.make_batch(64, spec, config=9, first=200)
    x = torch.from_numpy(frames).cuda()
    y = torch.full_like(x, -9.0)
    p = dc.params()
    dc.dc_complete_noalloc(x.data_ptr(), y.data_ptr(), 64, 32, 1024, p, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    for i in (0, 17, 63):
        _same(got[i], oracle.complete(frames[i]), False)


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
