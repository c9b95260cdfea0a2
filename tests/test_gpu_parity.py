"""GPU (libdc, sm_103a) against the CPU oracle, element by element.

Bar (arXiv 1802.00036, Section IV): bit-exact through the step-7 median --
steps 1-7a are selections and one float32 subtraction -- and within 1e-4 m
after the blur and the final inversion.  Every case calls the C-ABI through
the ctypes binding.
"""
import numpy as np
import pytest

import oracle
from paper_1802_00036_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_BLUR_M = 1e-4          # absolute, metres, after the Gaussian / bilateral
EXACT_STOPS = ["invert", "dilate", "close", "fill7", "extend", "fill_large", "median"]


@pytest.fixture(scope="module")
def ctx():
    from paper_1802_00036_gb300 import build, dc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = dc.Context(0)
    yield c
    c.close()


def gpu_run(ctx, frames, **kw):
    from paper_1802_00036_gb300 import dc
    x = torch.from_numpy(np.ascontiguousarray(frames, dtype=np.float32)).cuda()
    y = torch.full_like(x, -7.0)
    ctx.complete(x, y, dc.params(**kw))
    torch.cuda.synchronize()
    assert ctx.launches() >= 1
    return y.cpu().numpy()


def compare(got, want, stop, what=""):
    if stop in ("full", "blur"):
        err = np.abs(got.astype(np.float64) - want.astype(np.float64))
        assert err.max() <= TOL_BLUR_M, f"{what} max err {err.max()} at {np.unravel_index(err.argmax(), err.shape)}"
    else:
        bad = np.argwhere(got.view(np.uint32) != want.view(np.uint32))
        assert len(bad) == 0, f"{what} {len(bad)} mismatches, first {bad[:5].tolist()}"


SMALL = synth.FrameSpec(96, 200, 16, 0.05, 2.0, 80.0)


@pytest.mark.parametrize("stop", EXACT_STOPS + ["blur", "full"])
def test_every_stop_small_frames(ctx, stop):
    frames = np.stack([synth.make_frame(SMALL, 500 + i) for i in range(3)])
    got = gpu_run(ctx, frames, stop_after=stop)
    for i in range(3):
        compare(got[i], oracle.complete(frames[i], stop_after=stop), stop, f"frame {i}")


@pytest.mark.parametrize("shape", ["diamond5", "full5", "cross5", "full3", "circle5", "full7"])
@pytest.mark.parametrize("stop", ["dilate", "fill7", "median"])
def test_first_kernel_shapes(ctx, shape, stop):
    f = synth.make_frame(SMALL, 77)
    compare(gpu_run(ctx, f[None], first_kernel=shape, stop_after=stop)[0],
            oracle.complete(f, first_kernel=shape, stop_after=stop), stop, shape)


@pytest.mark.parametrize("quantize", [False, True])
@pytest.mark.parametrize("large", [3, 5, 15, 31, 51, 63])
def test_large_fill_sizes(ctx, large, quantize):
    # nearly empty maps: most tiles go to the step-6 worklist (on keys when
    # the depths are in 1/256 m steps, else on floats), every window size
    # from the smallest block of the window maxima to the largest
    f = synth.random_sparse(120, 170, 0.004, 31 + large, quantize=quantize)
    for stop in ("fill_large", "median", "full"):
        compare(gpu_run(ctx, f[None], large_fill=large, stop_after=stop)[0],
                oracle.complete(f, large_fill=large, stop_after=stop), stop, f"large {large}")


@pytest.mark.parametrize("quantize", [False, True])
@pytest.mark.parametrize("hole", [14, 22, 44])
@pytest.mark.parametrize("large", [15, 31, 51])
def test_large_fill_holes(ctx, hole, large, quantize):
    # a dense map with square holes: after steps 1-5 a hole of side s keeps
    # roughly (s - 6)^2 empty pixels, so small holes take the per-pixel fill
    # inside the main stage-B pass and large ones the worklist pass (on keys
    # when the depths are in 1/256 m steps, else on floats)
    f = synth.random_sparse(150, 250, 1.0, 3 + hole, 2.0, 80.0, quantize=quantize)
    for (y, x) in ((60, 40), (95, 130), (70, 200), (140, 5), (3, 246)):
        f[max(0, y - hole // 2):y + hole // 2, max(0, x - hole // 2):x + hole // 2] = 0.0
    for stop in ("fill_large", "median", "full"):
        compare(gpu_run(ctx, f[None], large_fill=large, stop_after=stop)[0],
                oracle.complete(f, large_fill=large, stop_after=stop), stop, f"hole {hole} large {large}")


def _step6_box(f, ty, tx, radius=15):
    """For the stage-B tile at (ty, tx): its empty pixels after step 5 (from
    the oracle) and the sizes of the step-6 scratch over them: the row
    maxima (box rows x distinct empty columns) and the box width."""
    E = oracle.complete(f, stop_after="extend")
    H, W = E.shape
    y0, x0 = ty - 4, tx - 4
    ys, xs = np.nonzero(E[max(0, y0):min(H, y0 + 68), max(0, x0):min(W, x0 + 68)] < 0.1)
    ys, xs = ys + max(0, y0), xs + max(0, x0)
    rows = min(H - 1, ys.max() + radius) - max(0, ys.min() - radius) + 1
    cols = min(W - 1, xs.max() + radius) - max(0, xs.min() - radius) + 1
    return len(ys), rows * len(set(xs.tolist())), cols


# Step-6 scratch of a stage-B CTA (floats): without and with the key buffer;
# a tile uses it when rows x distinct columns + 3 x box width fits.
SMALL_SCRATCH, BIG_SCRATCH = 3840, 6288


@pytest.mark.parametrize("layout", ["banded", "keys_rebuilt", "per_pixel"])
def test_step6_scattered_empties(ctx, layout):
    # holes cut in a dense map keep a core of empty pixels after steps 1-5
    # (a 13 x 13 hole about 3 x 3, an 11-row slot one row); placed in one
    # tile's region they give a sparse set of empties that the tile fills
    # itself: in bands through the small scratch (few distinct columns),
    # through the scratch that takes the keys' buffer (many columns; keys
    # rebuilt afterwards), or one warp per pixel when neither fits
    rects = {
        "banded": [(62, 75, 64, 77), (62, 75, 104, 117), (104, 117, 64, 77)],
        "keys_rebuilt": [(60, 71, 58, 118), (110, 121, 58, 118)],
        "per_pixel": [(52, 63, 50, 130), (116, 127, 50, 130)],
    }[layout]
    f = synth.random_sparse(180, 250, 1.0, 5, 2.0, 80.0)
    for (y0, y1, x0, x1) in rects:
        f[y0:y1, x0:x1] = 0.0
    n, rm, bc = _step6_box(f, 60, 60)
    assert 0 < n <= 160
    want = ("banded" if rm + 3 * bc <= SMALL_SCRATCH else "keys_rebuilt" if rm + 3 * bc <= BIG_SCRATCH
            else "per_pixel")
    assert want == layout, (n, rm, bc)
    for stop in ("fill_large", "median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop)[0], oracle.complete(f, stop_after=stop), stop, layout)


@pytest.mark.parametrize("layout", ["banded", "keys_rebuilt", "per_pixel"])
@pytest.mark.parametrize("off_grid_near", [False, True])
def test_step6_scattered_empties_on_keys(ctx, layout, off_grid_near):
    # the same holes in a map of 1/256 m depths: the tile fills them on keys
    # (the box through the idle region buffer, or one warp per pixel).  With
    # off-grid depths placed beside the holes, a value the fill reads may be
    # off the key grid: that tile then runs on floats instead
    rects = {
        "banded": [(62, 75, 64, 77), (62, 75, 104, 117), (104, 117, 64, 77)],
        "keys_rebuilt": [(60, 71, 58, 118), (110, 121, 58, 118)],
        "per_pixel": [(52, 63, 50, 130), (116, 127, 50, 130)],
    }[layout]
    f = synth.random_sparse(180, 250, 1.0, 5, 2.0, 80.0, quantize=True)
    for (y0, y1, x0, x1) in rects:
        f[y0:y1, x0:x1] = 0.0
        if off_grid_near:
            for (y, x) in ((y0 - 12, x0 - 12), (y1 + 11, x1 + 11), ((y0 + y1) // 2, x0 - 14)):
                if 0 <= y < f.shape[0] and 0 <= x < f.shape[1]:
                    f[y, x] = 50.0 + 1.0 / 1000
    for stop in ("fill_large", "median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop)[0], oracle.complete(f, stop_after=stop), stop, layout)


def _mixed_grid_frame(seed):
    """A 32-beam frame of 1/256 m depths in which one rectangle of depths is
    moved off that grid: the tiles that see it run on floats, the others on
    keys, in one call."""
    f = synth.make_frame(synth.FrameSpec(200, 400, 32, 0.06, 2.0, 80.0), seed)
    sub = f[110:170, 130:250]
    sub[sub > 0] += 1.0 / 1024
    return f


@pytest.mark.parametrize("stop", ["fill7", "extend", "fill_large", "median", "blur", "full"])
def test_grid_and_off_grid_tiles_in_one_frame(ctx, stop):
    frames = np.stack([_mixed_grid_frame(4321), synth.make_frame(synth.FrameSpec(200, 400, 32, 0.06), 17),
                       _mixed_grid_frame(99)])
    got = gpu_run(ctx, frames, stop_after=stop)
    for i in range(len(frames)):
        compare(got[i], oracle.complete(frames[i], stop_after=stop), stop, f"mixed {i}")


def test_off_grid_column_tops(ctx):
    # the topmost return of every seventh column moved off the 1/256 m grid:
    # step 5 copies off-grid values up those columns (and, after steps 2-4,
    # their neighbours), from the float map
    f = synth.make_frame(SMALL, 91)
    for x in range(0, SMALL.W, 7):
        ys = np.nonzero(f[:, x])[0]
        if len(ys):
            f[ys[0], x] += 1.0 / 512 + 1.0 / 4096
    for stop in ("extend", "fill_large", "median", "full"):
        for variant in (dict(), dict(extend_rows=6)):
            compare(gpu_run(ctx, f[None], stop_after=stop, **variant)[0],
                    oracle.complete(f, stop_after=stop, **variant), stop, f"tops {variant}")


@pytest.mark.parametrize("blur", ["gauss", "bilateral", "none"])
@pytest.mark.parametrize("median", [True, False])
def test_blur_variants(ctx, blur, median):
    f = synth.make_frame(synth.FrameSpec(150, 260, 32, 0.06, 1.0, 90.0), 11)
    for stop in ("blur", "full"):
        compare(gpu_run(ctx, f[None], blur=blur, median=median, stop_after=stop)[0],
                oracle.complete(f, blur=blur, median=median, stop_after=stop), stop, blur)


@pytest.mark.parametrize("variant", [dict(extend_top=False), dict(large_fill_on=False),
                                     dict(extend_rows=5), dict(extend_rows=0),
                                     dict(extend_top=False, large_fill_on=False)])
def test_point_cloud_variants(ctx, variant):
    f = synth.make_frame(SMALL, 123)
    for stop in ("median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop, **variant)[0],
                oracle.complete(f, stop_after=stop, **variant), stop, str(variant))


@pytest.mark.parametrize("large", [31, 51])
def test_capped_extension_with_scattered_off_grid_depths(ctx, large):
    # the extension capped at 50 rows sends the upper tiles to step 6's
    # worklist (run by the main pass itself for windows that fit its shared
    # memory, 31 here, else by the worklist kernel, 51); depths moved off the
    # key grid at random put some tiles, or only some tiles' wide step-6
    # regions, off the grid: those move on to the float passes
    f = synth.make_frame(synth.ONE_FRAME, synth.frame_seed(2, 9))
    rng = np.random.default_rng(17)
    ys, xs = np.nonzero(f > 0)
    pick = rng.choice(len(ys), max(1, len(ys) // 50), replace=False)
    f[ys[pick], xs[pick]] += np.float32(1.0 / 1024)
    for stop in ("fill_large", "median", "full"):
        compare(gpu_run(ctx, f[None], extend_rows=50, large_fill=large, stop_after=stop)[0],
                oracle.complete(f, extend_rows=50, large_fill=large, stop_after=stop), stop,
                f"capped, off-grid, large {large}")


@pytest.mark.parametrize("variant", [dict(extend_top=False, large_fill_on=False),
                                     dict(extend_rows=5, large_fill_on=False),
                                     dict(extend_top=False), dict(extend_rows=50),
                                     dict(extend_rows=20, large_fill=51)])
@pytest.mark.parametrize("lone_point", [False, True])
def test_empty_regions(ctx, variant, lone_point):
    # full-size frames whose upper third holds no return: without step 5 (or
    # with it capped) whole tiles, or the wide windows of step 6, see only
    # empty values; a lone return near the top makes the tiles around its
    # column differ from their neighbours
    frames = synth.make_batch(2, synth.ONE_FRAME, config=11)
    if lone_point:
        frames[0, 8, 610] = 37.5
        frames[1, 70, 3] = 12.25
    got = gpu_run(ctx, frames, **variant)
    for stop in ("fill_large", "median", "full"):
        if stop != "full":
            got_s = gpu_run(ctx, frames, stop_after=stop, **variant)
        for i in range(2):
            compare(got[i] if stop == "full" else got_s[i],
                    oracle.complete(frames[i], stop_after=stop, **variant), stop, f"{variant} frame {i}")


@pytest.mark.parametrize("quantize", [False, True])
@pytest.mark.parametrize("hw", [(1, 1), (1, 37), (41, 1), (2, 2), (3, 5), (7, 64), (33, 65),
                                (64, 128), (65, 129), (5, 300)])
def test_edge_shapes(ctx, hw, quantize):
    # quantised: every tile on keys (the key box crosses the frame's edges);
    # otherwise on floats
    f = synth.random_sparse(*hw, 0.2, hw[0] * 1000 + hw[1], quantize=quantize)
    for stop in ("fill7", "extend", "median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop)[0], oracle.complete(f, stop_after=stop),
                stop, str(hw))


@pytest.mark.parametrize("fill", ["empty", "dense", "top_only", "one_point"])
def test_degenerate_frames(ctx, fill):
    H, W = 70, 140
    f = np.zeros((H, W), np.float32)
    if fill == "dense":
        f = synth.random_sparse(H, W, 1.0, 5, 1.0, 80.0)
    elif fill == "top_only":
        f[0, :] = 12.5
    elif fill == "one_point":
        f[50, 70] = 33.0
    for stop in ("fill7", "median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop)[0], oracle.complete(f, stop_after=stop),
                stop, fill)


def test_out_of_range_inputs_follow_the_formulas(ctx):
    # depths >= 100 m invert to values <= 0 (empty); tiny depths are empty
    f = synth.random_sparse(40, 90, 0.3, 8, 0.0, 130.0)
    f[5, 5] = 100.0
    f[6, 6] = 0.05
    for stop in ("fill7", "median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop)[0], oracle.complete(f, stop_after=stop),
                stop, "range")


@pytest.mark.parametrize("extreme", [100.0, 99.95703125, 100.5, 0.09765625])
def test_quantised_depths_at_the_key_range_ends(ctx, extreme):
    # depths in 1/256 m steps with one extreme value: 100 m inverts to 0 and
    # (256 d) - 25600 = 0 is still a key; just below 100 m inverts to a
    # non-empty-looking but empty value; above 100 m inverts below 0, which
    # no key holds (that unit runs on floats); just below 0.1 m is empty
    f = synth.random_sparse(90, 300, 0.1, 17, 2.0, 80.0, quantize=True)
    f[40, 150] = extreme
    f[80, 20] = extreme
    for stop in ("fill7", "median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop)[0], oracle.complete(f, stop_after=stop),
                stop, f"extreme {extreme}")


def test_full_size_frame_352x1216(ctx):
    f = synth.make_frame(synth.ONE_FRAME, synth.frame_seed(0, 0))
    for stop in ("fill7", "median", "full"):
        compare(gpu_run(ctx, f[None], stop_after=stop)[0], oracle.complete(f, stop_after=stop),
                stop, "352x1216")


@pytest.mark.parametrize("stop", ["blur", "full"])
def test_quantised_frames_bit_exact_through_the_blur(ctx, stop):
    # depths in steps of 1/256 m (KITTI's fixed point): every tile runs on
    # 16-bit keys and the Gaussian is summed exactly, so the whole chain --
    # blur and final inversion included -- equals the oracle bit for bit
    frames = [synth.make_frame(synth.ONE_FRAME, synth.frame_seed(0, 1)),
              synth.make_frame(SMALL, 777)]
    for f in frames:
        assert np.array_equal(np.rint(f * 256.0) / 256.0, f)
        got = gpu_run(ctx, f[None], stop_after=stop)[0]
        want = oracle.complete(f, stop_after=stop)
        bad = np.argwhere(got.view(np.uint32) != want.view(np.uint32))
        assert len(bad) == 0, f"{len(bad)} mismatches, first {bad[:5].tolist()}"


def test_batched_375x1242_sampled_and_batch_independent(ctx):
    # the 64-frame batched workload; three frames checked against the oracle,
    # every frame checked against its own single-frame run
    n = 64
    frames = synth.make_batch(n, synth.UNIFORM_375, config=1, density_range=(0.04, 0.06))
    for stop in ("median", "full"):
        got = gpu_run(ctx, frames, stop_after=stop)
        for i in (0, 31, 63):
            compare(got[i], oracle.complete(frames[i], stop_after=stop), stop, f"frame {i}")
        for i in range(0, n, 9):
            alone = gpu_run(ctx, frames[i:i + 1], stop_after=stop)[0]
            assert np.array_equal(alone.view(np.uint32), got[i].view(np.uint32)), i


def test_bench_workload_sampled(ctx):
    # the benchmark's own batch: 64 frames of 352x1216 (its seeds), one call
    # in its launch shape (16 stage-A warps per SM, 5 stage-B CTAs per SM,
    # step-6 threshold 160; one shape, so the region arrives by tensor copy);
    # the depths are 1/256 m steps, so sampled frames equal the oracle bit for
    # bit through the blur, and every eighth frame equals its own run alone
    from paper_1802_00036_gb300 import dc
    frames = synth.make_batch(64, synth.ONE_FRAME, config=0)
    dc.dc_set_tuning(ctx.h, 16, 5, 160)
    try:
        got = gpu_run(ctx, frames)
        for i in (0, 21, 42, 63):
            want = oracle.complete(frames[i])
            bad = np.argwhere(got[i].view(np.uint32) != want.view(np.uint32))
            assert len(bad) == 0, f"frame {i}: {len(bad)} mismatches, first {bad[:5].tolist()}"
        for i in range(0, 64, 8):
            alone = gpu_run(ctx, frames[i:i + 1])[0]
            assert np.array_equal(alone.view(np.uint32), got[i].view(np.uint32)), i
    finally:
        dc.dc_set_tuning(ctx.h, 8, 5, 160)


def test_bilateral_full_size(ctx):
    f = synth.make_frame(synth.UNIFORM_375, synth.frame_seed(1, 3))
    compare(gpu_run(ctx, f[None], blur="bilateral")[0], oracle.complete(f, blur="bilateral"),
            "full", "bilateral")


def test_uneven_batch_one_call(ctx):
    from paper_1802_00036_gb300 import dc
    specs = [synth.MIX[i % 4] for i in range(8)]
    host = [synth.make_frame(s, synth.frame_seed(2, i)) for i, s in enumerate(specs)]
    ins = [torch.from_numpy(h).cuda() for h in host]
    # the third frame's output lives in a wider buffer (pitch > W)
    outs = []
    for i, h in enumerate(host):
        buf = torch.full((h.shape[0], h.shape[1] + (24 if i == 2 else 0)), -3.0, device="cuda")
        outs.append(buf[:, :h.shape[1]])
    for stop in ("median", "full"):
        ctx.complete_frames(list(zip(ins, outs)), dc.params(stop_after=stop))
        torch.cuda.synchronize()
        for i in (0, 1, 2, 3, 6):
            compare(outs[i].cpu().numpy(), oracle.complete(host[i], stop_after=stop), stop, f"mix {i}")


@pytest.mark.parametrize("variant", [dict(extend_rows=20), dict(extend_top=False)])
def test_uneven_batch_capped_extension(ctx, variant):
    # frames of four shapes in one call (regions by cp.async, tiles frame by
    # frame) with the extension capped or off: the tiles with many empty
    # pixels run the step-6 worklist's code inside the main pass
    from paper_1802_00036_gb300 import dc
    specs = [synth.MIX[i % 4] for i in range(4)]
    host = [synth.make_frame(s, synth.frame_seed(3, i)) for i, s in enumerate(specs)]
    ins = [torch.from_numpy(h).cuda() for h in host]
    outs = [torch.full_like(x, -3.0) for x in ins]
    for stop in ("fill_large", "full"):
        ctx.complete_frames(list(zip(ins, outs)), dc.params(stop_after=stop, **variant))
        torch.cuda.synchronize()
        for i in range(4):
            compare(outs[i].cpu().numpy(), oracle.complete(host[i], stop_after=stop, **variant), stop,
                    f"mix {i} {variant}")


@pytest.mark.parametrize("kw,want", [
    (dict(), 5),                                   # frame table, stage A, stage B and both step-6 lists
    (dict(extend_rows=20), 4),                     # worklist tiles inside stage B: no worklist kernel
    (dict(extend_top=False), 4),
    (dict(extend_rows=20, large_fill=51), 5),      # a 51 x 51 window's region does not fit there
    (dict(large_fill_on=False), 3),                # no step 6: no step-6 kernels
    (dict(stop_after="extend"), 3),
    (dict(stop_after="fill7"), 2),                 # stage A on floats writes the output
])
def test_kernels_launched_per_call(ctx, kw, want):
    # the launch sequence of one call (dc_last_launch_count), each variant
    # still giving the oracle's result
    f = synth.make_frame(SMALL, 321)
    got = gpu_run(ctx, f[None], **kw)[0]
    assert ctx.launches() == want
    stop = kw.get("stop_after", "full")
    compare(got, oracle.complete(f, **kw), stop, str(kw))


def test_per_size_tunings_in_a_mixed_call(ctx):
    # step-6 thresholds recorded per frame size apply to those frames in a
    # call that mixes sizes; the results stay the oracle's
    from paper_1802_00036_gb300 import dc
    specs = [synth.MIX[i % 4] for i in range(4)]
    host = [synth.make_frame(s, synth.frame_seed(4, i)) for i, s in enumerate(specs)]
    ins = [torch.from_numpy(h).cuda() for h in host]
    outs = [torch.full_like(x, -3.0) for x in ins]
    try:
        for i, s in enumerate(specs):
            dc.dc_set_class_tuning(ctx.h, s.H, s.W, (8, 5, (0, 8, 160, 32)[i], 128))
        ctx.complete_frames(list(zip(ins, outs)), dc.params(extend_rows=20))
        torch.cuda.synchronize()
        for i in range(4):
            compare(outs[i].cpu().numpy(), oracle.complete(host[i], extend_rows=20), "full", f"mix {i}")
        with pytest.raises(dc.DcError):
            dc.dc_set_class_tuning(ctx.h, 10, 10, (8, 5, 161, 128))
        with pytest.raises(dc.DcError):
            dc.dc_set_class_tuning(ctx.h, 0, 10, (8, 5, 16, 128))
        dc.dc_set_class_tuning(ctx.h, 0, 0, None)
        for k in range(16):  # the table holds 16 sizes
            dc.dc_set_class_tuning(ctx.h, 10 + k, 10, (8, 5, 16, 128))
        with pytest.raises(dc.DcError) as e:
            dc.dc_set_class_tuning(ctx.h, 99, 10, (8, 5, 16, 128))
        assert e.value.status == 5
    finally:
        dc.dc_set_class_tuning(ctx.h, 0, 0, None)


def test_host_buffers_entry_point(ctx):
    from paper_1802_00036_gb300 import dc
    frames = np.stack([synth.make_frame(SMALL, 900 + i) for i in range(4)])
    out = np.full_like(frames, -1.0)
    dc.dc_complete_host(ctx.h, frames.ctypes.data, out.ctypes.data, 4, SMALL.H, SMALL.W, dc.params())
    dev = gpu_run(ctx, frames)
    assert np.array_equal(out.view(np.uint32), dev.view(np.uint32))


def test_host_buffers_pipelined_chunks(ctx):
    # 20 full-size frames: the copies and kernels run in three overlapped chunks
    from paper_1802_00036_gb300 import dc
    frames = synth.make_batch(20, synth.ONE_FRAME, config=7)
    hin = torch.from_numpy(frames).pin_memory()
    hout = torch.full_like(hin, -1.0).pin_memory()
    dc.dc_complete_host(ctx.h, hin.data_ptr(), hout.data_ptr(), 20, 352, 1216, dc.params())
    dev = gpu_run(ctx, frames)
    assert np.array_equal(hout.numpy().view(np.uint32), dev.view(np.uint32))


def test_host_buffers_async_stream_of_batches(ctx):
    # five calls in flight before one wait: the two staging sets are each
    # reused while earlier calls' copies may still run; every batch must
    # come back as the device path computes it (one of them of another size)
    from paper_1802_00036_gb300 import dc
    sizes = (12, 12, 5, 12, 12)
    batches = [synth.make_batch(n, synth.ONE_FRAME, config=8, first=10 * i) for i, n in enumerate(sizes)]
    hins = [torch.from_numpy(b).pin_memory() for b in batches]
    houts = [torch.full_like(h, -1.0).pin_memory() for h in hins]
    stream = torch.cuda.Stream()
    for h_in, h_out, n in zip(hins, houts, sizes):
        dc.dc_complete_host_async(ctx.h, h_in.data_ptr(), h_out.data_ptr(), n, 352, 1216, dc.params(),
                                  stream.cuda_stream)
    dc.dc_host_wait(ctx.h)
    for b, h_out in zip(batches, houts):
        assert np.array_equal(h_out.numpy().view(np.uint32), gpu_run(ctx, b).view(np.uint32))
    with pytest.raises(dc.DcError):
        dc.dc_complete_host_async(ctx.h, 0, 0, 1, 352, 1216, dc.params())


def test_host_calls_interleaved_with_device_calls(ctx):
    # host-buffer calls run their kernels on a stream of the context; a
    # device-buffer call on another stream in between shares the scratch and
    # must be ordered after them, and the next host call after it
    from paper_1802_00036_gb300 import dc
    b0, b1, b2 = (synth.make_batch(8, synth.ONE_FRAME, config=9, first=10 * i) for i in range(3))
    h0, h2 = torch.from_numpy(b0).pin_memory(), torch.from_numpy(b2).pin_memory()
    o0, o2 = torch.full_like(h0, -1.0).pin_memory(), torch.full_like(h2, -1.0).pin_memory()
    x1 = torch.from_numpy(b1).cuda()
    y1 = torch.full_like(x1, -1.0)
    other = torch.cuda.Stream()
    torch.cuda.synchronize()
    dc.dc_complete_host_async(ctx.h, h0.data_ptr(), o0.data_ptr(), 8, 352, 1216, dc.params())
    dc.dc_complete_uniform(ctx.h, x1.data_ptr(), y1.data_ptr(), 8, 352, 1216, dc.params(), other.cuda_stream)
    dc.dc_complete_host_async(ctx.h, h2.data_ptr(), o2.data_ptr(), 8, 352, 1216, dc.params(),
                              other.cuda_stream)
    dc.dc_host_wait(ctx.h)
    other.synchronize()
    for b, got in ((b0, o0.numpy()), (b1, y1.cpu().numpy()), (b2, o2.numpy())):
        assert np.array_equal(got.view(np.uint32), gpu_run(ctx, b).view(np.uint32))


def test_results_do_not_depend_on_tuning(ctx):
    from paper_1802_00036_gb300 import dc
    frames = synth.make_batch(6, synth.UNIFORM_375, config=4)
    x = torch.from_numpy(frames).cuda()
    ref = None
    for a, b, f, c in ((12, 3, 16, 128), (1, 1, 0, 64), (3, 2, 160, 128), (64, 1, 4, 64), (8, 4, 160, 128),
                       (2, 5, 8, 64), (16, 5, 160, 64), (8, 5, 160, 128)):
        dc.dc_set_tuning(ctx.h, a, b, f, c)
        y = torch.full_like(x, -2.0)
        ctx.complete(x, y)
        torch.cuda.synchronize()
        got = y.cpu().numpy().view(np.uint32)
        if ref is None:
            ref = got
        assert np.array_equal(got, ref), (a, b, f, c)
    y = torch.empty_like(x)
    a, b, f, c = dc.dc_autotune(ctx.h, x.data_ptr(), y.data_ptr(), 6, 375, 1242, dc.params())
    assert 1 <= a <= 64 and 1 <= b <= 5 and 0 <= f <= 160 and c in (64, 128)
    assert dc.dc_get_tuning(ctx.h) == (a, b, f, c)
    dc.dc_set_tuning(ctx.h, 8, 5, 160)
    with pytest.raises(dc.DcError):
        dc.dc_set_tuning(ctx.h, 0, 3)
    with pytest.raises(dc.DcError):
        dc.dc_set_tuning(ctx.h, 8, 5, 160, 96)


@pytest.mark.parametrize("shape", ["diamond5", "full5", "cross5", "full3", "circle5", "full7"])
@pytest.mark.parametrize("quantize", [False, True])
def test_narrow_strips_every_element(ctx, shape, quantize):
    # stage A in 64-column strips (two columns per lane) for every element, on
    # keys and (off-grid depths) on floats, the key kernel redoing the narrow
    # strips' units itself; frames wider than one strip with a ragged tail
    from paper_1802_00036_gb300 import dc
    f = synth.random_sparse(70, 233, 0.12, 61, quantize=quantize)
    dc.dc_set_tuning(ctx.h, 8, 5, 160, 64)
    try:
        for stop in ("extend", "median", "full"):
            compare(gpu_run(ctx, f[None], first_kernel=shape, stop_after=stop)[0],
                    oracle.complete(f, first_kernel=shape, stop_after=stop), stop, f"{shape} narrow")
    finally:
        dc.dc_set_tuning(ctx.h, 8, 5, 160)


def test_profiling_one_call_in_several(ctx):
    # every third call of seven is profiled (calls 0, 3 and 6), with both
    # stages timed; the results do not depend on it
    from paper_1802_00036_gb300 import dc
    frames = synth.make_batch(2, SMALL, config=12)
    x = torch.from_numpy(frames).cuda()
    want = gpu_run(ctx, frames)
    dc.dc_set_profiling(ctx.h, 3)
    try:
        for _ in range(7):
            y = torch.full_like(x, -1.0)
            ctx.complete(x, y)
        torch.cuda.synchronize()
        times = dc.dc_kernel_times(ctx.h)
        assert len(times) == 3 and all(a > 0 and b > 0 for a, b in times)
        assert np.array_equal(y.cpu().numpy().view(np.uint32), want.view(np.uint32))
    finally:
        dc.dc_set_profiling(ctx.h, 0)
    assert dc.dc_kernel_times(ctx.h) == []
    with pytest.raises(dc.DcError):
        dc.dc_set_profiling(ctx.h, -1)


def test_graph_cache_replays_calls(ctx):
    # with the cache on, a repeated call is one graph launch of the same
    # kernels: the same bits as without, the current contents of the same
    # buffers, other buffers captured anew, least recently used evicted,
    # profiled calls run directly, scratch growth drops the graphs, and a
    # call on another stream is still ordered after the previous one
    from paper_1802_00036_gb300 import dc
    spec = synth.FrameSpec(120, 250, 32, 0.05, 2.0, 80.0)
    sets = [synth.make_batch(3, spec, config=13, first=10 * k) for k in range(3)]
    want = [gpu_run(ctx, f) for f in sets]
    xs = [torch.from_numpy(f).cuda() for f in sets]
    ys = [torch.empty_like(x) for x in xs]
    p = dc.params()
    st = torch.cuda.current_stream().cuda_stream
    launches = None

    def call(k, stream=st):
        ys[k].fill_(-3.0)
        if stream != st:
            torch.cuda.synchronize()          # the fill above ran on the current stream
        dc.dc_complete_uniform(ctx.h, xs[k].data_ptr(), ys[k].data_ptr(), 3, spec.H, spec.W, p, stream)

    def check(k, expect):
        torch.cuda.synchronize()
        assert np.array_equal(ys[k].cpu().numpy().view(np.uint32), expect.view(np.uint32)), k

    dc.dc_set_graph_cache(ctx.h, 2)
    try:
        for rep in range(3):                  # capture, then replays
            call(0)
            check(0, want[0])
            if launches is None:
                launches = ctx.launches()
            assert ctx.launches() == launches
            assert dc.dc_graph_cache_entries(ctx.h) == 1
        xs[0].copy_(xs[1])                    # new contents, same buffers
        call(0)
        check(0, want[1])
        xs[0].copy_(torch.from_numpy(sets[0]).cuda())
        for k in (1, 2, 0, 1):                # three buffer sets through two graphs
            call(k)
            check(k, want[k])
            assert dc.dc_graph_cache_entries(ctx.h) == 2
        other = torch.cuda.Stream()
        call(2, other.cuda_stream)            # ordered after the call before it
        other.synchronize()
        check(2, want[2])
        dc.dc_set_profiling(ctx.h, 1)         # profiled calls are not captured
        dc.dc_set_graph_cache(ctx.h, 3)       # (a new size drops the graphs)
        assert dc.dc_graph_cache_entries(ctx.h) == 0
        call(1)
        check(1, want[1])
        assert dc.dc_graph_cache_entries(ctx.h) == 0
        assert len(dc.dc_kernel_times(ctx.h)) == 1
        dc.dc_set_profiling(ctx.h, 0)
        big = synth.make_batch(40, synth.ONE_FRAME, config=13)
        got_big = gpu_run(ctx, big)            # may grow the scratch: the graphs go
        assert np.array_equal(got_big[5].view(np.uint32), gpu_run(ctx, big[5:6])[0].view(np.uint32))
        for k in (0, 1):
            call(k)
            check(k, want[k])
        assert dc.dc_graph_cache_entries(ctx.h) >= 1
    finally:
        dc.dc_set_graph_cache(ctx.h, 0)
        dc.dc_set_profiling(ctx.h, 0)
    assert dc.dc_graph_cache_entries(ctx.h) == 0
    for bad in (-1, dc.DC_MAX_GRAPHS + 1):
        with pytest.raises(dc.DcError):
            dc.dc_set_graph_cache(ctx.h, bad)


def test_graph_cache_with_host_buffer_calls(ctx):
    # a stream of host-buffer calls replays the graphs of its chunks (two
    # staging sets x two chunks) and returns every batch as computed directly
    from paper_1802_00036_gb300 import dc
    batches = [synth.make_batch(16, synth.ONE_FRAME, config=14, first=20 * i) for i in range(5)]
    want = [gpu_run(ctx, b) for b in batches]
    hins = [torch.from_numpy(b).pin_memory() for b in batches]
    houts = [torch.full_like(h, -1.0).pin_memory() for h in hins]
    dc.dc_set_graph_cache(ctx.h, 8)
    try:
        for h_in, h_out in zip(hins, houts):
            dc.dc_complete_host_async(ctx.h, h_in.data_ptr(), h_out.data_ptr(), 16, 352, 1216, dc.params())
        dc.dc_host_wait(ctx.h)
        assert dc.dc_graph_cache_entries(ctx.h) == 4
    finally:
        dc.dc_set_graph_cache(ctx.h, 0)
    for w, h_out in zip(want, houts):
        assert np.array_equal(h_out.numpy().view(np.uint32), w.view(np.uint32))


def test_invalid_arguments_are_refused(ctx):
    from paper_1802_00036_gb300 import dc
    x = torch.zeros((2, 16, 16), device="cuda")
    y = torch.zeros_like(x)
    p = dc.params()
    bad = [
        lambda: dc.dc_complete_uniform(ctx.h, 0, y.data_ptr(), 2, 16, 16, p),
        lambda: dc.dc_complete_uniform(ctx.h, x.data_ptr(), y.data_ptr(), 2, 0, 16, p),
        lambda: dc.dc_complete_uniform(ctx.h, x.data_ptr(), x.data_ptr(), 2, 16, 16, p),
        lambda: dc.dc_complete_uniform(ctx.h, x.data_ptr(), x.data_ptr() + 1024, 2, 16, 16, p),
        lambda: dc.dc_complete(ctx.h, [(x.data_ptr(), y.data_ptr(), 16, 16, 8, 16)], p),
        lambda: dc.dc_complete_uniform(ctx.h, x.data_ptr(), y.data_ptr(), 2, 16, 16,
                                       dc.params(large_fill=30)),
        lambda: dc.dc_complete_uniform(ctx.h, x.data_ptr(), y.data_ptr(), 2, 16, 16,
                                       dc.params(first_kernel=9)),
        lambda: dc.dc_complete_uniform(ctx.h, x.data_ptr(), y.data_ptr(), 2, 16, 16,
                                       dc.params(blur="bilateral", sigma_color=0.0)),
    ]
    for i, call in enumerate(bad):
        with pytest.raises(dc.DcError) as e:
            call()
        assert e.value.status == 1, i
    # nothing was queued and the context still works
    assert dc.dc_last_async_error(ctx.h) == 0
    dc.dc_complete_uniform(ctx.h, x.data_ptr(), y.data_ptr(), 2, 16, 16, p)
    torch.cuda.synchronize()


def test_zero_frames_is_a_no_op(ctx):
    from paper_1802_00036_gb300 import dc
    dc.dc_complete(ctx.h, [], dc.params())
    assert ctx.launches() == 0


def test_scratch_budget_is_enforced(ctx):
    from paper_1802_00036_gb300 import dc
    small = dc.Context(0, scratch_budget_bytes=64 * 1024)
    try:
        x = torch.zeros((4, 352, 1216), device="cuda")
        with pytest.raises(dc.DcError) as e:
            small.complete(x)
        assert e.value.status == 2
    finally:
        small.close()
