"""Seeded synthetic sparse LIDAR depth maps (stand-in for KITTI depth completion).

The paper evaluates on KITTI depth completion (Section V): LIDAR scans
projected into the image plane, giving a sparse map the size of the image in
which only the lower two thirds hold points, at 5-7% density there, with
depths up to 80 m.  KITTI is not available here, so frames are drawn from a
seeded synthetic scene with that structure:

* a pinhole camera 1.7 m above a ground plane, optical axis level;
* 20 axis-aligned boxes standing on the ground (cars, walls, poles, trees);
* B horizontal scan lines ("beams") spread over the lower two thirds of the
  frame, each with a smooth +-1 row wobble along the columns;
* each beam pixel returns the ray-cast depth of the scene with a per-beam
  column probability chosen so that the valid fraction of the *whole frame*
  is the target density; rays that hit nothing, or land outside
  [d_min, d_max], return nothing (0);
* 1% of returns are replaced by uniform outliers in [d_min, d_max];
* depths are optionally quantised to 1/256 m (KITTI's storage resolution).

Random numbers come from a counter-based splitmix64 stream written here, so a
frame depends only on its seed, on every machine and numpy version.  This
module holds none of the depth-completion arithmetic; it only makes inputs.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

CAMERA_HEIGHT_M = 1.7
N_BOXES = 20


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based uniform stream: value i of stream (seed, tag) is
    mix64(key + (i + 1) * golden) with key = mix64(seed * golden + tag)."""

    def __init__(self, seed: int, tag: int):
        with np.errstate(over="ignore"):
            base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(tag & 0xFFFFFFFF)
        self.key = _mix64(np.array([base], dtype=np.uint64))[0]
        self.count = 0

    def uniform(self, shape, lo=0.0, hi=1.0) -> np.ndarray:
        n = int(np.prod(shape)) if shape != () else 1
        idx = np.arange(self.count + 1, self.count + 1 + n, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            u = _mix64(self.key + idx * _GOLDEN)
        x = (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return (lo + (hi - lo) * x).reshape(shape)


@dataclasses.dataclass(frozen=True)
class FrameSpec:
    """One synthetic frame: size, beams, target density and depth range."""
    H: int = 352
    W: int = 1216
    beams: int = 64
    density: float = 0.05
    d_min: float = 2.0
    d_max: float = 80.0
    outlier_frac: float = 0.01
    quantize: bool = True


def _camera(spec: FrameSpec):
    f = 0.58 * spec.W          # ~ KITTI's 721 px focal length at W = 1242
    cx = 0.5 * spec.W
    cy = 0.43 * spec.H         # horizon a little above mid-frame
    return f, cx, cy


def _boxes(rng: Stream):
    """N_BOXES boxes standing on the ground: columns x0,x1,y0,y1,z0,z1 (m)."""
    cx = rng.uniform((N_BOXES,), -16.0, 16.0)
    z0 = rng.uniform((N_BOXES,), 4.0, 60.0)
    w = rng.uniform((N_BOXES,), 0.4, 4.0)
    h = rng.uniform((N_BOXES,), 0.6, 9.0)
    d = rng.uniform((N_BOXES,), 0.4, 5.0)
    y1 = np.full(N_BOXES, CAMERA_HEIGHT_M)          # camera y axis points down
    return np.stack([cx - w / 2, cx + w / 2, y1 - h, y1, z0, z0 + d], axis=1)


def _ray_depth(u: np.ndarray, v: np.ndarray, spec: FrameSpec, boxes: np.ndarray) -> np.ndarray:
    """Z-depth of the first surface along the rays through pixel centres
    (u, v); inf where the ray hits nothing."""
    f, cx, cy = _camera(spec)
    dx = (u + 0.5 - cx) / f
    dy = (v + 0.5 - cy) / f
    depth = np.full(u.shape, np.inf)
    ground = dy > 1e-9
    depth[ground] = CAMERA_HEIGHT_M / dy[ground]
    # slab test, ray = t * (dx, dy, 1): t is the z-depth
    with np.errstate(divide="ignore", invalid="ignore"):
        for x0, x1, y0, y1, z0, z1 in boxes:
            tx0, tx1 = x0 / dx, x1 / dx
            ty0, ty1 = y0 / dy, y1 / dy
            tn = np.maximum.reduce([np.minimum(tx0, tx1), np.minimum(ty0, ty1),
                                    np.full(u.shape, z0)])
            tf = np.minimum.reduce([np.maximum(tx0, tx1), np.maximum(ty0, ty1),
                                    np.full(u.shape, z1)])
            hit = (tn <= tf) & (tf > 0) & np.isfinite(tn)
            depth = np.where(hit & (tn < depth), tn, depth)
    return depth


def ground_truth(spec: FrameSpec, seed: int) -> np.ndarray:
    """Dense ray-cast depth of the frame's scene (0 where out of range)."""
    rng = Stream(seed, 1)
    boxes = _boxes(rng)
    v, u = np.mgrid[0:spec.H, 0:spec.W].astype(np.float64)
    d = _ray_depth(u.ravel(), v.ravel(), spec, boxes).reshape(spec.H, spec.W)
    d[(d < spec.d_min) | (d > spec.d_max) | ~np.isfinite(d)] = 0.0
    return d.astype(np.float32)


def make_frame(spec: FrameSpec, seed: int) -> np.ndarray:
    """One sparse H x W float32 depth map (0 = empty) for ``seed``."""
    H, W, B = spec.H, spec.W, max(1, spec.beams)
    boxes = _boxes(Stream(seed, 1))
    rng = Stream(seed, 2)
    # beam rows: evenly over the lower two thirds, smooth wobble of +-1 row
    phase = rng.uniform((B,), 0.0, 2.0 * np.pi)
    period = rng.uniform((B,), 150.0, 400.0)
    cols = np.arange(W, dtype=np.float64)
    base = H / 3.0 + (np.arange(B) + 0.5) * (2.0 * H / 3.0) / B
    rows = np.rint(base[:, None] + np.sin(2.0 * np.pi * cols[None, :] / period[:, None]
                                          + phase[:, None]))
    rows = np.clip(rows, 0, H - 1).astype(np.int64)
    uu = np.broadcast_to(cols[None, :], rows.shape)
    depth = _ray_depth(uu.ravel(), rows.astype(np.float64).ravel(), spec, boxes).reshape(rows.shape)
    ok = (depth >= spec.d_min) & (depth <= spec.d_max)
    # per-beam column probability giving the target whole-frame density
    target = spec.density * H * W
    usable = max(int(ok.sum()), 1)
    p = min(1.0, target / usable)
    keep = ok & (rng.uniform(rows.shape) < p)
    vals = depth.copy()
    out_u = rng.uniform(rows.shape)
    out_v = rng.uniform(rows.shape, spec.d_min, spec.d_max)
    vals = np.where(out_u < spec.outlier_frac, out_v, vals)
    if spec.quantize:
        vals = np.maximum(np.rint(vals * 256.0) / 256.0, spec.d_min)
    frame = np.zeros((H, W), dtype=np.float32)
    r, c = rows[keep], uu[keep].astype(np.int64)
    v = vals[keep].astype(np.float32)
    # beams may collide on a row after the wobble: keep the nearest return
    order = np.argsort(-v, kind="stable")
    frame[r[order], c[order]] = v[order]
    return frame


def frame_seed(config: int, frame: int) -> int:
    return 1802000 + config * 1000 + frame


def make_batch(n: int, spec: FrameSpec, config: int = 1, first: int = 0,
               density_range: tuple[float, float] | None = None) -> np.ndarray:
    """(n, H, W) float32 frames; with ``density_range`` each frame draws its
    own density uniformly from it (the 4-6% batched workload)."""
    out = np.empty((n, spec.H, spec.W), dtype=np.float32)
    for i in range(n):
        seed = frame_seed(config, first + i)
        s = spec
        if density_range is not None:
            lo, hi = density_range
            dens = float(Stream(seed, 3).uniform(()) * (hi - lo) + lo)
            s = dataclasses.replace(spec, density=dens)
        out[i] = make_frame(s, seed)
    return out


# Named workloads (shapes, densities and depth ranges of the paper's data).
ONE_FRAME = FrameSpec(352, 1216, 64, 0.05, 2.0, 80.0)
UNIFORM_375 = FrameSpec(375, 1242, 64, 0.05, 1.0, 90.0)
MIX = (
    FrameSpec(256, 512, 32, 0.03, 2.0, 80.0),
    FrameSpec(352, 1216, 64, 0.05, 2.0, 80.0),
    FrameSpec(375, 1242, 64, 0.05, 2.0, 80.0),
    FrameSpec(512, 2048, 128, 0.10, 2.0, 80.0),
)


def random_sparse(H: int, W: int, density: float, seed: int, d_min=0.5, d_max=99.0,
                  quantize: bool = False) -> np.ndarray:
    """Unstructured sparse map (uniform positions and depths) for edge cases."""
    rng = Stream(seed, 7)
    keep = rng.uniform((H, W)) < density
    vals = rng.uniform((H, W), d_min, d_max)
    if quantize:
        vals = np.rint(vals * 256.0) / 256.0
    return np.where(keep, vals, 0.0).astype(np.float32)


def camera_matrix(spec: FrameSpec) -> np.ndarray:
    """3 x 4 projection of the synthetic camera (pixel centres at +0.5)."""
    f, cx, cy = _camera(spec)
    return np.array([[f, 0.0, cx, 0.0], [0.0, f, cy, 0.0], [0.0, 0.0, 1.0, 0.0]])


def point_cloud(spec: FrameSpec, seed: int, extra: int = 20000) -> np.ndarray:
    """N x 3 float32 camera-frame points: every return of `make_frame`
    lifted to 3D at its pixel centre, plus `extra` points behind the camera,
    outside the field of view or beyond the depth range."""
    frame = make_frame(spec, seed)
    f, cx, cy = _camera(spec)
    r, c = np.nonzero(frame)
    z = frame[r, c].astype(np.float64)
    x = (c + 0.5 - cx) / f * z
    y = (r + 0.5 - cy) / f * z
    pts = np.stack([x, y, z], axis=1)
    rng = Stream(seed, 9)
    far = rng.uniform((extra, 3), -120.0, 120.0)
    pts = np.concatenate([pts, far])
    order = np.argsort(rng.uniform((len(pts),)))
    return pts[order].astype(np.float32)
