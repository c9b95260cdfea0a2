"""Continuous-batching depth-completion server on one GPU (Python side).

`NativeServer` wraps libdc's own server (dc_server_*): a C++ worker thread
keeps a fixed pool of device slots sized by a memory budget, admits a
submitted frame when a slot is free (otherwise the frame waits:
back-pressure), copies it into its slot, closes a batch when it holds
`max_batch` ready frames or when the oldest one has waited `deadline_ms`,
runs it as ONE `dc_complete` call on one of `lanes` in-flight lanes (each
with its own libdc context and CUDA stream), copies the results back and
reports each frame's tag and latency.  `drive_native` replays Poisson
arrivals of several sensors into it.

Every step of the chain runs in libdc's kernels; this module only submits
frames and keeps time.  The per-frame arithmetic does not depend on the
batch a frame lands in, so results are the same alone and in the mix.
"""
from __future__ import annotations

import gc
import time

import numpy as np

from . import dc


def poisson_schedule(rate_hz: float, sensors: int, seconds: float, seed: int = 0) -> np.ndarray:
    """Sorted arrival times (s) and sensor ids of `sensors` Poisson streams
    of `rate_hz` each over `seconds`."""
    rng = np.random.default_rng(seed)
    times, ids = [], []
    for s in range(sensors):
        n = rng.poisson(rate_hz * seconds)
        times.append(np.sort(rng.uniform(0.0, seconds, n)))
        ids.append(np.full(n, s))
    t = np.concatenate(times)
    i = np.concatenate(ids)
    order = np.argsort(t, kind="stable")
    return t[order], i[order]


class NativeServer:
    """libdc's serving worker (dc_server_create / submit / poll / destroy):
    frames up to `max_hw`, device slots from `budget_bytes`, batches of up
    to `max_batch` closed at `deadline_ms`, `lanes` contexts and streams.
    Input and output buffers are host memory (pinned for asynchronous
    copies); a frame's buffers stay untouched until its tag is polled."""

    def __init__(self, max_hw=(512, 2048), budget_bytes=2 << 30, deadline_ms=2.0, max_batch=64, lanes=3,
                 device=0, params=None):
        self.max_hw = max_hw
        self.h = dc.dc_server_create(device, max_hw[0], max_hw[1], int(budget_bytes), int(round(deadline_ms * 1e3)),
                                     int(max_batch), int(lanes), params if params is not None else dc.params())
        self._poll = dc.poll_buffers(4096)

    def submit(self, host_in: int, host_out: int, H: int, W: int, tag: int) -> None:
        dc.dc_server_submit(self.h, host_in, host_out, H, W, tag)

    def poll(self):
        return dc.dc_server_poll(self.h, 4096, self._poll)

    def stats(self) -> dict:
        return dc.dc_server_get_stats(self.h)

    def close(self):
        if self.h:
            dc.dc_server_destroy(self.h)
            self.h = None


def drive_native(server: NativeServer, frames_by_sensor, rate_hz: float, seconds: float, seed: int = 0,
                 outstanding: int = 128) -> dict:
    """Replay Poisson arrivals of every sensor at `rate_hz` into `server`.
    frames_by_sensor: per sensor a list of pinned (H, W) float32 tensors,
    re-used round-robin.  Results go to a ring of `outstanding` pinned
    buffers; when all of them are in flight the next arrival waits for one.
    A frame's latency runs from its scheduled arrival to its result in host
    memory (the wait before submission included)."""
    import torch
    times, ids = poisson_schedule(rate_hz, len(frames_by_sensor), seconds, seed)
    Hm, Wm = server.max_hw
    outs = [torch.empty((Hm, Wm)).pin_memory() for _ in range(outstanding)]
    out_ptrs = [o.data_ptr() for o in outs]
    pools = [[(f.data_ptr(), f.shape[0], f.shape[1]) for f in pool] for pool in frames_by_sensor]
    free = list(range(outstanding))
    in_flight = {}
    lat = []
    counters = [0] * len(frames_by_sensor)
    b0 = server.stats()["batches"]
    t_last = None

    def collect():
        nonlocal t_last
        got = server.poll()
        if got:
            now = time.perf_counter()
            for tag, ms in got:
                b, due, sub = in_flight.pop(tag)
                lat.append((sub - due) * 1e3 + ms)
                free.append(b)
            t_last = now
        return len(got)

    # no collection pauses in the client while it keeps the schedule (one in
    # a large process's heap delays a submission by tens of milliseconds)
    gc_was_on = gc.isenabled()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for k, (t, s) in enumerate(zip(times, ids)):
            due = t0 + t
            while True:
                now = time.perf_counter()
                if now >= due and free:
                    break
                if not collect() and due - now > 1e-4:
                    time.sleep(min(due - now, 1e-3) * 0.5)
            pool = pools[s]
            ptr, H, W = pool[counters[s] % len(pool)]
            counters[s] += 1
            b = free.pop()
            in_flight[k] = (b, due, time.perf_counter())
            server.submit(ptr, out_ptrs[b], H, W, k)
        while in_flight:
            if not collect():
                time.sleep(5e-5)
    finally:
        if gc_was_on:
            gc.enable()
    n = len(lat)
    span = max((t_last or t0) - (t0 + (times[0] if n else 0.0)), 1e-9)
    arr = np.array(lat) if lat else np.zeros(1)
    batches = server.stats()["batches"] - b0
    return {"frames": n, "frames_per_s": n / span, "p50_ms": float(np.percentile(arr, 50)),
            "p99_ms": float(np.percentile(arr, 99)), "mean_batch": n / max(batches, 1), "batches": batches,
            "offered_hz": rate_hz * len(frames_by_sensor)}
