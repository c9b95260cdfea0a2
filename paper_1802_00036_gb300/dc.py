"""Thin ctypes binding of libdc (include/dc.h).

Functions carry the C names and only marshal arguments: every step of the
depth-completion chain runs in the CUDA kernels of ``lib/libdc.so``.  There is
no CPU fallback: if the library is missing or no GPU is present, calls raise.

PyTorch is used by callers only for device memory and streams; tensors are
passed as raw device pointers (``tensor.data_ptr()``) and streams as
``torch.cuda.Stream.cuda_stream`` integers.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libdc.so")

DC_OK = 0
DC_ERR_INVALID_ARG, DC_ERR_OOM, DC_ERR_CUDA, DC_ERR_TIMEOUT, DC_ERR_UNSUPPORTED = 1, 2, 3, 4, 5
STATUS = {0: "DC_OK", 1: "DC_ERR_INVALID_ARG", 2: "DC_ERR_OOM", 3: "DC_ERR_CUDA",
          4: "DC_ERR_TIMEOUT", 5: "DC_ERR_UNSUPPORTED"}
KERNELS = {"diamond5": 0, "full5": 1, "cross5": 2, "full3": 3, "circle5": 4, "full7": 5}
BLURS = {"none": 0, "gauss": 1, "bilateral": 2}
STOPS = {"full": 0, "invert": 1, "dilate": 2, "close": 3, "fill7": 4, "extend": 5,
         "fill_large": 6, "median": 7, "blur": 8}


class DcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class dc_params(ctypes.Structure):
    _fields_ = [
        ("first_kernel", ctypes.c_int),
        ("large_fill", ctypes.c_int),
        ("median", ctypes.c_int),
        ("blur", ctypes.c_int),
        ("sigma_space", ctypes.c_float),
        ("sigma_color", ctypes.c_float),
        ("extend_top", ctypes.c_int),
        ("extend_rows", ctypes.c_int),
        ("large_fill_on", ctypes.c_int),
        ("stop_after", ctypes.c_int),
    ]


class dc_tuning(ctypes.Structure):
    _fields_ = [("a_warps_per_sm", ctypes.c_int), ("b_ctas_per_sm", ctypes.c_int),
                ("b_sparse_fill", ctypes.c_int), ("a_strip_cols", ctypes.c_int)]


class dc_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("done", ctypes.c_ulonglong),
                ("batches", ctypes.c_ulonglong), ("slots", ctypes.c_int), ("lanes", ctypes.c_int)]


class dc_frame(ctypes.Structure):
    _fields_ = [
        ("in_", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("H", ctypes.c_int),
        ("W", ctypes.c_int),
        ("in_pitch", ctypes.c_int),
        ("out_pitch", ctypes.c_int),
    ]


_lib = None

# (name, restype, argtypes) for every symbol include/dc.h declares
SIGNATURES = [
    ("dc_params_default", ctypes.c_int, [ctypes.POINTER(dc_params)]),
    ("dc_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]),
    ("dc_complete", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dc_frame), ctypes.c_int,
                                   ctypes.POINTER(dc_params), ctypes.c_void_p]),
    ("dc_complete_uniform", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(dc_params), ctypes.c_void_p]),
    ("dc_complete_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(dc_params), ctypes.c_void_p]),
    ("dc_complete_host_async", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(dc_params), ctypes.c_void_p]),
    ("dc_host_wait", ctypes.c_int, [ctypes.c_void_p]),
    ("dc_reserve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("dc_last_launch_count", ctypes.c_int, [ctypes.c_void_p]),
    ("dc_project", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("dc_metrics", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("dc_set_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dc_tuning)]),
    ("dc_set_class_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(dc_tuning)]),
    ("dc_get_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dc_tuning)]),
    ("dc_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(dc_params), ctypes.c_void_p,
                                   ctypes.POINTER(dc_tuning)]),
    ("dc_set_profiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("dc_set_graph_cache", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("dc_graph_cache_entries", ctypes.c_int, [ctypes.c_void_p]),
    ("dc_kernel_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    ("dc_last_async_error", ctypes.c_int, [ctypes.c_void_p]),
    ("dc_inject_fault", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("dc_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("dc_destroy", None, [ctypes.c_void_p]),
    ("dc_complete_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.POINTER(dc_params), ctypes.c_void_p]),
    ("dc_server_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(dc_params)]),
    ("dc_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_ulonglong]),
    ("dc_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("dc_server_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(dc_server_stats)]),
    ("dc_server_destroy", None, [ctypes.c_void_p]),
]


def load(path: str = LIB_PATH):
    """Load libdc.so (built by ``paper_1802_00036_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libdc.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, what: str):
    if status != DC_OK:
        raise DcError(status, what)


def params(first_kernel="diamond5", large_fill=31, median=True, blur="gauss", sigma_space=1.5,
           sigma_color=0.5, extend_top=True, extend_rows=-1, large_fill_on=True,
           stop_after="full") -> dc_params:
    """dc_params from keywords; defaults are the paper's final design."""
    p = dc_params()
    _check(load().dc_params_default(ctypes.byref(p)), "dc_params_default")
    p.first_kernel = KERNELS[first_kernel] if isinstance(first_kernel, str) else int(first_kernel)
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


def dc_params_default() -> dc_params:
    p = dc_params()
    _check(load().dc_params_default(ctypes.byref(p)), "dc_params_default")
    return p


def dc_create(device: int = 0, scratch_budget_bytes: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().dc_create(ctypes.byref(h), int(device), int(scratch_budget_bytes)), "dc_create")
    return h


def dc_destroy(ctx) -> None:
    if ctx:
        load().dc_destroy(ctx)


def dc_complete(ctx, frames, p: dc_params, stream: int = 0) -> None:
    """frames: sequence of (in_ptr, out_ptr, H, W, in_pitch, out_pitch)."""
    arr = (dc_frame * max(1, len(frames)))()
    for i, (a, b, H, W, ip, op) in enumerate(frames):
        arr[i] = dc_frame(a, b, H, W, ip, op)
    _check(load().dc_complete(ctx, arr, len(frames), ctypes.byref(p), ctypes.c_void_p(stream)),
           "dc_complete")


def dc_complete_uniform(ctx, in_ptr: int, out_ptr: int, n: int, H: int, W: int, p: dc_params,
                        stream: int = 0) -> None:
    _check(load().dc_complete_uniform(ctx, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), n, H, W,
                                      ctypes.byref(p), ctypes.c_void_p(stream)), "dc_complete_uniform")


def dc_complete_host(ctx, host_in: int, host_out: int, n: int, H: int, W: int, p: dc_params,
                     stream: int = 0) -> None:
    _check(load().dc_complete_host(ctx, ctypes.c_void_p(host_in), ctypes.c_void_p(host_out), n, H, W,
                                   ctypes.byref(p), ctypes.c_void_p(stream)), "dc_complete_host")


def dc_complete_host_async(ctx, host_in: int, host_out: int, n: int, H: int, W: int, p: dc_params,
                           stream: int = 0) -> None:
    _check(load().dc_complete_host_async(ctx, ctypes.c_void_p(host_in), ctypes.c_void_p(host_out), n, H, W,
                                         ctypes.byref(p), ctypes.c_void_p(stream)), "dc_complete_host_async")


def dc_host_wait(ctx) -> None:
    _check(load().dc_host_wait(ctx), "dc_host_wait")


def dc_server_create(device: int, max_H: int, max_W: int, budget_bytes: int, deadline_us: int, max_batch: int,
                     lanes: int, p: dc_params) -> int:
    h = ctypes.c_void_p()
    _check(load().dc_server_create(ctypes.byref(h), device, max_H, max_W, budget_bytes, deadline_us, max_batch,
                                   lanes, ctypes.byref(p)), "dc_server_create")
    return h.value


def dc_server_submit(srv, host_in: int, host_out: int, H: int, W: int, tag: int) -> None:
    _check(load().dc_server_submit(srv, ctypes.c_void_p(host_in), ctypes.c_void_p(host_out), H, W, tag),
           "dc_server_submit")


def poll_buffers(max_n: int = 4096):
    """Tag and latency arrays for dc_server_poll, to be reused across polls."""
    return (ctypes.c_ulonglong * max_n)(), (ctypes.c_double * max_n)()


def dc_server_poll(srv, max_n: int = 4096, buffers=None):
    """[(tag, latency_ms), ...] of the frames done since the last poll (at
    most max_n; `buffers` from poll_buffers(max_n) saves allocating them)."""
    tags, lat = buffers if buffers is not None else poll_buffers(max_n)
    n = ctypes.c_int()
    _check(load().dc_server_poll(srv, tags, lat, max_n, ctypes.byref(n)), "dc_server_poll")
    return [(tags[i], lat[i]) for i in range(n.value)]


def dc_server_get_stats(srv) -> dict:
    st = dc_server_stats()
    _check(load().dc_server_get_stats(srv, ctypes.byref(st)), "dc_server_get_stats")
    return {"submitted": st.submitted, "done": st.done, "batches": st.batches, "slots": st.slots,
            "lanes": st.lanes}


def dc_server_destroy(srv) -> None:
    if srv:
        load().dc_server_destroy(srv)


def dc_complete_noalloc(in_ptr: int, out_ptr: int, n: int, H: int, W: int, p: dc_params,
                        stream: int = 0) -> None:
    """Context-free call that allocates no device memory: its scratch is a
    fixed array inside the library, shared by every call (see include/dc.h
    for the limits and for why overlapping calls race)."""
    _check(load().dc_complete_noalloc(ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), n, H, W,
                                      ctypes.byref(p), ctypes.c_void_p(stream)), "dc_complete_noalloc")


def dc_reserve(ctx, n_frames: int, H: int, W: int) -> None:
    _check(load().dc_reserve(ctx, n_frames, H, W), "dc_reserve")


def dc_project(ctx, xyz_ptr: int, n_points: int, P, H: int, W: int, d_min: float, d_max: float,
               depth_ptr: int, pitch: int | None = None, stream: int = 0) -> None:
    """Nearest-depth projection of device points (N x 3 float32) into a
    device H x W map; P: 12 numbers (3 x 4, row-major)."""
    pm = (ctypes.c_double * 12)(*[float(v) for v in list(P)])
    _check(load().dc_project(ctx, ctypes.c_void_p(xyz_ptr), int(n_points), pm, H, W, float(d_min), float(d_max),
                             ctypes.c_void_p(depth_ptr), W if pitch is None else int(pitch),
                             ctypes.c_void_p(stream)), "dc_project")


def dc_metrics(ctx, pred_ptr: int, gt_ptr: int, n: int, H: int, W: int, stream: int = 0):
    """[(rmse_mm, mae_mm, irmse_per_km, imae_per_km, valid), ...] per frame."""
    out = (ctypes.c_double * (5 * max(1, n)))()
    _check(load().dc_metrics(ctx, ctypes.c_void_p(pred_ptr), ctypes.c_void_p(gt_ptr), n, H, W, out,
                             ctypes.c_void_p(stream)), "dc_metrics")
    return [tuple(out[5 * i:5 * i + 5]) for i in range(n)]


def dc_set_tuning(ctx, a_warps_per_sm: int, b_ctas_per_sm: int, b_sparse_fill: int = 160,
                  a_strip_cols: int = 128) -> None:
    t = dc_tuning(int(a_warps_per_sm), int(b_ctas_per_sm), int(b_sparse_fill), int(a_strip_cols))
    _check(load().dc_set_tuning(ctx, ctypes.byref(t)), "dc_set_tuning")


def dc_set_class_tuning(ctx, H: int, W: int, tuning=None) -> None:
    """Record `tuning` (a_warps_per_sm, b_ctas_per_sm, b_sparse_fill,
    a_strip_cols) for frames of H x W; None forgets every size."""
    if tuning is None:
        _check(load().dc_set_class_tuning(ctx, int(H), int(W), None), "dc_set_class_tuning")
        return
    t = dc_tuning(*(int(v) for v in tuning))
    _check(load().dc_set_class_tuning(ctx, int(H), int(W), ctypes.byref(t)), "dc_set_class_tuning")


def dc_get_tuning(ctx) -> tuple[int, int, int, int]:
    t = dc_tuning()
    _check(load().dc_get_tuning(ctx, ctypes.byref(t)), "dc_get_tuning")
    return t.a_warps_per_sm, t.b_ctas_per_sm, t.b_sparse_fill, t.a_strip_cols


def dc_autotune(ctx, in_ptr: int, out_ptr: int, n: int, H: int, W: int, p: dc_params,
                stream: int = 0) -> tuple[int, int, int, int]:
    t = dc_tuning()
    _check(load().dc_autotune(ctx, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), n, H, W, ctypes.byref(p),
                              ctypes.c_void_p(stream), ctypes.byref(t)), "dc_autotune")
    return t.a_warps_per_sm, t.b_ctas_per_sm, t.b_sparse_fill, t.a_strip_cols


def dc_last_launch_count(ctx) -> int:
    return int(load().dc_last_launch_count(ctx))


DC_PROFILE_CALLS = 4096
DC_MAX_GRAPHS = 64


def dc_set_graph_cache(ctx, max_graphs: int) -> None:
    """Replay repeated calls from up to `max_graphs` CUDA graphs (0: off)."""
    _check(load().dc_set_graph_cache(ctx, int(max_graphs)), "dc_set_graph_cache")


def dc_graph_cache_entries(ctx) -> int:
    return int(load().dc_graph_cache_entries(ctx))


def dc_set_profiling(ctx, every) -> None:
    """Profile one call in `every` (True: every call; False or 0: off)."""
    every = int(every) if not isinstance(every, bool) else int(every)
    _check(load().dc_set_profiling(ctx, every), "dc_set_profiling")


def dc_kernel_times(ctx, max_calls: int = DC_PROFILE_CALLS):
    """[(stage_a_ms, stage_b_ms), ...] for the last profiled calls, oldest first."""
    buf = (ctypes.c_float * (2 * max(1, max_calls)))()
    n = ctypes.c_int()
    _check(load().dc_kernel_times(ctx, buf, int(max_calls), ctypes.byref(n)), "dc_kernel_times")
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(n.value)]


def dc_last_async_error(ctx) -> int:
    return int(load().dc_last_async_error(ctx))


DC_FAULT_WAIT, DC_FAULT_LAUNCH = 1, 2


def dc_inject_fault(ctx, fault: int) -> None:
    """Testing hook (see include/dc.h): leave the context as a device-side
    wait timeout (DC_FAULT_WAIT) or a refused launch (DC_FAULT_LAUNCH) would."""
    _check(load().dc_inject_fault(ctx, int(fault)), "dc_inject_fault")


def dc_status_str(s: int) -> str:
    return load().dc_status_str(int(s)).decode()


class Context:
    """Owns one dc_ctx; helpers take torch CUDA tensors."""

    def __init__(self, device: int = 0, scratch_budget_bytes: int = 0):
        self.device = device
        self.h = dc_create(device, scratch_budget_bytes)

    def close(self):
        if self.h:
            dc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream) -> int:
        if stream is None:
            import torch
            return torch.cuda.current_stream().cuda_stream
        return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream

    def complete(self, inp, out=None, p: dc_params | None = None, stream=None):
        """inp: (n, H, W) or (H, W) float32 CUDA tensor, contiguous."""
        import torch
        if inp.dtype != torch.float32 or not inp.is_cuda or not inp.is_contiguous():
            raise ValueError("expected a contiguous float32 CUDA tensor")
        x = inp if inp.dim() == 3 else inp.unsqueeze(0)
        if out is None:
            out = torch.empty_like(inp)
        y = out if out.dim() == 3 else out.unsqueeze(0)
        dc_complete_uniform(self.h, x.data_ptr(), y.data_ptr(), x.shape[0], x.shape[1], x.shape[2],
                            p if p is not None else params(), self._stream(stream))
        return out

    def complete_frames(self, pairs, p: dc_params | None = None, stream=None):
        """pairs: list of (in, out) 2-D float32 CUDA tensors of any sizes (row-major,
        unit column stride); all frames run in one call."""
        fr = []
        for a, b in pairs:
            fr.append((a.data_ptr(), b.data_ptr(), a.shape[0], a.shape[1], a.stride(0), b.stride(0)))
        dc_complete(self.h, fr, p if p is not None else params(), self._stream(stream))

    def launches(self) -> int:
        return dc_last_launch_count(self.h)
