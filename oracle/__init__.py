"""CPU oracle for the depth-completion chain of arXiv 1802.00036, Section IV.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, single-threaded C
statement of the eight steps (``dco.c``).  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the
GPU library never does, and the two share no code.

``build()`` compiles ``libdco.so`` next to this file with the host C compiler.
Each wrapper takes and returns numpy arrays; float maps are float32 H x W.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dco.c")
_LIB = os.path.join(_HERE, "libdco.so")

# Codes mirror oracle/dco.h.
SHAPES = {"diamond5": 0, "full5": 1, "cross5": 2, "full3": 3, "circle5": 4, "full7": 5}
BLURS = {"none": 0, "gauss": 1, "bilateral": 2}
STOPS = {"full": 0, "invert": 1, "dilate": 2, "close": 3, "fill7": 4,
         "extend": 5, "fill_large": 6, "median": 7, "blur": 8}

_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    """Mirror of ``dco_params`` (oracle/dco.h)."""
    _fields_ = [
        ("first_kernel", ctypes.c_int),
        ("large_fill", ctypes.c_int),
        ("median", ctypes.c_int),
        ("blur", ctypes.c_int),
        ("sigma_space", ctypes.c_double),
        ("sigma_color", ctypes.c_double),
        ("extend_top", ctypes.c_int),
        ("extend_rows", ctypes.c_int),
        ("large_fill_on", ctypes.c_int),
        ("stop_after", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile libdco.so (plain C, -O2, no fast-math) if it is missing or stale."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "dco.h"))))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                   "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        f = ctypes.POINTER(ctypes.c_float)
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        sig = {
            "dco_complete": [f, f, i, i, ctypes.POINTER(Params)],
            "dco_invert": [f, f, i, i],
            "dco_dilate_shape": [f, f, i, i, i],
            "dco_dilate_square": [f, f, i, i, i],
            "dco_erode_square": [f, f, i, i, i],
            "dco_close_square": [f, f, i, i, i],
            "dco_fill_square": [f, f, i, i, i],
            "dco_extend_top": [f, f, i, i, i],
            "dco_median5": [f, f, i, i],
            "dco_gauss5": [f, d, i, i],
            "dco_bilateral5": [f, d, i, i, ctypes.c_double, ctypes.c_double],
            "dco_metrics": [f, f, i, i, d],
            "dco_project": [f, ctypes.c_long, d, i, i, ctypes.c_double, ctypes.c_double, f],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.dco_params_default.argtypes = [ctypes.POINTER(Params)]
        lib.dco_params_default.restype = None
        _lib = lib
    return _lib


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_map(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("expected an H x W map")
    return a


def params(first_kernel="diamond5", large_fill=31, median=True, blur="gauss",
           sigma_space=1.5, sigma_color=0.5, extend_top=True, extend_rows=-1,
           large_fill_on=True, stop_after="full") -> Params:
    """Build oracle parameters; defaults are the paper's final design."""
    p = Params()
    _load().dco_params_default(ctypes.byref(p))
    p.first_kernel = SHAPES[first_kernel] if isinstance(first_kernel, str) else int(first_kernel)
    p.large_fill = int(large_fill)
    p.median = int(bool(median))
    p.blur = BLURS[blur] if isinstance(blur, str) else int(blur)
    p.sigma_space = float(sigma_space)
    p.sigma_color = float(sigma_color)
    p.extend_top = int(bool(extend_top))
    p.extend_rows = int(extend_rows)
    p.large_fill_on = int(bool(large_fill_on))
    p.stop_after = STOPS[stop_after] if isinstance(stop_after, str) else int(stop_after)
    return p


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def complete(depth, **kw) -> np.ndarray:
    """Run the whole chain (Section IV, steps 1-8) on one H x W float32 map."""
    a = _as_map(depth)
    out = np.empty_like(a)
    p = params(**kw)
    _check(_load().dco_complete(_fptr(a), _fptr(out), a.shape[0], a.shape[1], ctypes.byref(p)),
           "complete")
    return out


def complete_batch(frames, **kw) -> np.ndarray:
    """Run ``complete`` frame by frame over an (n, H, W) stack."""
    frames = np.asarray(frames, dtype=np.float32)
    return np.stack([complete(f, **kw) for f in frames]) if len(frames) else frames.copy()


def _unary(name, a, *extra):
    a = _as_map(a)
    out = np.empty_like(a)
    _check(getattr(_load(), name)(_fptr(a), _fptr(out), a.shape[0], a.shape[1], *extra), name)
    return out


def invert(d):
    """Step 1: 100 - d on non-empty pixels, 0 elsewhere."""
    return _unary("dco_invert", d)


def dilate_shape(a, shape):
    return _unary("dco_dilate_shape", a, SHAPES[shape] if isinstance(shape, str) else int(shape))


def dilate_square(a, k):
    return _unary("dco_dilate_square", a, int(k))


def erode_square(a, k):
    return _unary("dco_erode_square", a, int(k))


def close_square(a, k):
    return _unary("dco_close_square", a, int(k))


def fill_square(a, k):
    return _unary("dco_fill_square", a, int(k))


def extend_top(c, max_rows=-1):
    return _unary("dco_extend_top", c, int(max_rows))


def median5(f):
    return _unary("dco_median5", f)


def gauss5(m) -> np.ndarray:
    m = _as_map(m)
    g = np.empty(m.shape, dtype=np.float64)
    _check(_load().dco_gauss5(_fptr(m), _dptr(g), m.shape[0], m.shape[1]), "gauss5")
    return g


def bilateral5(m, sigma_space=1.5, sigma_color=0.5) -> np.ndarray:
    m = _as_map(m)
    g = np.empty(m.shape, dtype=np.float64)
    _check(_load().dco_bilateral5(_fptr(m), _dptr(g), m.shape[0], m.shape[1],
                                  float(sigma_space), float(sigma_color)), "bilateral5")
    return g


def metrics(pred, gt) -> dict:
    """KITTI-style accuracy of `pred` against `gt` (H x W, metres)."""
    p, g = _as_map(pred), _as_map(gt)
    if p.shape != g.shape:
        raise ValueError("shape mismatch")
    out = np.zeros(5, dtype=np.float64)
    _check(_load().dco_metrics(_fptr(p), _fptr(g), p.shape[0], p.shape[1], _dptr(out)), "metrics")
    return {"rmse_mm": out[0], "mae_mm": out[1], "irmse_per_km": out[2], "imae_per_km": out[3],
            "valid": int(out[4])}


def project(xyz, P, H: int, W: int, d_min: float = 0.1, d_max: float = 1e30) -> np.ndarray:
    """Nearest depth per pixel of the points `xyz` (N x 3) under the 3 x 4
    projection `P` (Section V: scans projected with the camera calibration)."""
    pts = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    Pm = np.ascontiguousarray(P, dtype=np.float64).reshape(12)
    out = np.empty((H, W), dtype=np.float32)
    _check(_load().dco_project(_fptr(pts), len(pts), _dptr(Pm), H, W, float(d_min), float(d_max), _fptr(out)),
           "project")
    return out
