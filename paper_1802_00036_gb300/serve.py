"""Continuous-batching depth-completion server on one GPU.

Two forms of the same server.  `NativeServer` is libdc's own (dc_server_*):
a C++ worker thread admits, batches, copies and completes, and Python only
submits frames and collects their tags and latencies (`drive_native`).
`Server` below is the same design in Python threads, kept as a readable
statement of it; its own threads bound its throughput to a few thousand
frames per second.

Frames arrive from sensors (host arrays, any of the configured sizes).  The
server keeps a fixed pool of device slots sized by a memory budget; a frame
is admitted when a slot is free (otherwise it waits: back-pressure), copied
into its slot on an upload stream, and becomes ready.  A batcher closes a
batch when it holds `max_batch` ready frames or when the oldest one has
waited `deadline_ms`, and runs it as ONE `dc_complete` call (frames of mixed
sizes, each with its slot's row pitch) on one of `lanes` in-flight lanes --
each lane owns its own libdc context and CUDA stream, so a batch can run
while the next one is being formed and launched.  When a batch's kernels
finish, its outputs are copied back to pinned host buffers, the slots return
to the pool, and every frame's latency (arrival to result on the host) is
recorded.

Every step of the chain runs in libdc's kernels; this module only moves
frames, batches them and keeps time.  The per-frame arithmetic does not
depend on the batch a frame lands in, so results are the same alone and in
the mix.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import dc


@dataclasses.dataclass
class _Req:
    frame: np.ndarray          # host float32 H x W (pinned or not)
    arrival: float             # perf_counter seconds
    future: Future
    slot: int = -1
    ready_event: object = None
    sensor: int = 0


@dataclasses.dataclass
class Stats:
    latencies_ms: list
    completed: int
    started: float
    finished: float
    batches: int

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        span = max(self.finished - self.started, 1e-9)
        return {"frames": self.completed, "frames_per_s": self.completed / span,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_batch": self.completed / max(self.batches, 1), "batches": self.batches}


class Server:
    """Continuous batching of depth-completion requests on one GPU."""

    def __init__(self, max_hw=(512, 2048), budget_bytes=2 << 30, deadline_ms=2.0, max_batch=64,
                 lanes=3, device=0, params=None, copy_results=True):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.Hmax, self.Wmax = max_hw
        slot_bytes = 2 * self.Hmax * self.Wmax * 4          # input + output
        scratch_per_lane = max_batch * (self.Hmax * ((self.Wmax + 31) // 32 * 32) + self.Wmax) * 4
        avail = budget_bytes - lanes * scratch_per_lane
        self.n_slots = max(1, min(4096, avail // slot_bytes))
        self.d_in = torch.empty((self.n_slots, self.Hmax, self.Wmax), device=self.device)
        self.d_out = torch.empty_like(self.d_in)
        self.h_out = torch.empty((self.n_slots, self.Hmax, self.Wmax), pin_memory=True)
        self.free = queue.Queue()
        for i in range(self.n_slots):
            self.free.put(i)
        self.copy_results = copy_results
        self.deadline = deadline_ms / 1e3
        self.max_batch = max_batch
        self.params = params if params is not None else dc.params()
        self.upload = torch.cuda.Stream(self.device)
        self.lanes = []
        for _ in range(lanes):
            ctx = dc.Context(device, scratch_budget_bytes=scratch_per_lane + (64 << 20))
            dc.dc_reserve(ctx.h, max_batch, self.Hmax, self.Wmax)
            self.lanes.append((ctx, torch.cuda.Stream(self.device), torch.cuda.Stream(self.device)))
        self.lane_free = queue.Queue()
        for i in range(lanes):
            self.lane_free.put(i)
        self.admit_q = queue.Queue()      # arrived, waiting for a slot
        self.ready_q = queue.Queue()      # uploaded, waiting for a batch
        self.done_q = queue.Queue()       # launched batches
        self.lock = threading.Lock()
        self.latencies = []
        self.completed = 0
        self.batches = 0
        self.t_first = None
        self.t_last = None
        self.stop = False
        self.threads = [threading.Thread(target=f, daemon=True)
                        for f in (self._admitter, self._batcher, self._completer)]
        for t in self.threads:
            t.start()

    # -- public -------------------------------------------------------------
    def submit(self, frame, sensor: int = 0, arrival: float | None = None) -> Future:
        """Queue one H x W float32 frame (numpy array, or a pinned CPU torch
        tensor for asynchronous upload); the future resolves to the output
        as a numpy array (None when the server was made with
        copy_results=False, e.g. to time serving alone)."""
        H, W = frame.shape
        if H > self.Hmax or W > self.Wmax:
            raise ValueError("frame larger than the server's slots")
        fut = Future()
        r = _Req(frame=frame, arrival=time.perf_counter() if arrival is None else arrival, future=fut,
                 sensor=sensor)
        self.admit_q.put(r)
        return fut

    def stats(self) -> Stats:
        with self.lock:
            return Stats(list(self.latencies), self.completed, self.t_first or 0.0, self.t_last or 0.0,
                         self.batches)

    def reset_stats(self):
        with self.lock:
            self.latencies = []
            self.completed = 0
            self.batches = 0
            self.t_first = None
            self.t_last = None

    def close(self):
        self.stop = True
        self.admit_q.put(None)
        self.ready_q.put(None)
        self.done_q.put(None)
        for t in self.threads:
            t.join(timeout=5)
        for ctx, _, _ in self.lanes:
            ctx.close()

    # -- internals ------------------------------------------------------------
    def _admitter(self):
        torch = self.torch
        while not self.stop:
            r = self.admit_q.get()
            if r is None:
                return
            r.slot = self.free.get()                  # back-pressure: waits for a slot
            H, W = r.frame.shape
            with torch.cuda.stream(self.upload):
                src = r.frame if isinstance(r.frame, torch.Tensor) else torch.from_numpy(r.frame)
                self.d_in[r.slot, :H, :W].copy_(src, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.upload)
            r.ready_event = ev
            self.ready_q.put(r)

    def _batcher(self):
        torch = self.torch
        pending = []
        while not self.stop:
            timeout = None
            if pending:
                timeout = max(0.0, pending[0].arrival + self.deadline - time.perf_counter())
            try:
                r = self.ready_q.get(timeout=timeout)
                if r is None:
                    return
                pending.append(r)
                if len(pending) < self.max_batch:
                    continue
            except queue.Empty:
                pass
            if not pending:
                continue
            batch, pending = pending[:self.max_batch], pending[self.max_batch:]
            lane = self.lane_free.get()
            ctx, stream, down = self.lanes[lane]
            for r in batch:
                stream.wait_event(r.ready_event)
            frames = []
            for r in batch:
                H, W = r.frame.shape
                frames.append((self.d_in[r.slot].data_ptr(), self.d_out[r.slot].data_ptr(), H, W,
                               self.Wmax, self.Wmax))
            dc.dc_complete(ctx.h, frames, self.params, stream.cuda_stream)
            ran = torch.cuda.Event()
            ran.record(stream)
            with torch.cuda.stream(down):
                down.wait_event(ran)
                for r in batch:
                    H, W = r.frame.shape
                    self.h_out[r.slot, :H, :W].copy_(self.d_out[r.slot, :H, :W], non_blocking=True)
                back = torch.cuda.Event()
                back.record(down)
            self.done_q.put((lane, batch, back))

    def _completer(self):
        while not self.stop:
            item = self.done_q.get()
            if item is None:
                return
            lane, batch, back = item
            back.synchronize()
            now = time.perf_counter()
            self.lane_free.put(lane)
            with self.lock:
                for r in batch:
                    self.latencies.append((now - r.arrival) * 1e3)
                self.completed += len(batch)
                self.batches += 1
                if self.t_first is None:
                    self.t_first = min(r.arrival for r in batch)
                self.t_last = now
            for r in batch:
                H, W = r.frame.shape
                res = self.h_out[r.slot, :H, :W].numpy().copy() if self.copy_results else None
                self.free.put(r.slot)
                r.future.set_result(res)


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


def drive(server: Server, frames_by_sensor, rate_hz: float, seconds: float, seed: int = 0) -> dict:
    """Replay Poisson arrivals of every sensor at `rate_hz` into `server`
    (frames are pre-built host arrays, re-used round-robin per sensor) and
    return the latency / throughput summary once every result is back."""
    times, ids = poisson_schedule(rate_hz, len(frames_by_sensor), seconds, seed)
    server.reset_stats()
    futs = []
    counters = [0] * len(frames_by_sensor)
    t0 = time.perf_counter()
    for t, s in zip(times, ids):
        due = t0 + t
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            if due - now > 2e-4:
                time.sleep((due - now) * 0.5)
        pool = frames_by_sensor[s]
        f = pool[counters[s] % len(pool)]
        counters[s] += 1
        futs.append(server.submit(f, sensor=int(s), arrival=due))
    for f in futs:
        f.result(timeout=60)
    out = server.stats().summary()
    out["offered_hz"] = rate_hz * len(frames_by_sensor)
    return out


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
    n = len(lat)
    span = max((t_last or t0) - (t0 + (times[0] if n else 0.0)), 1e-9)
    arr = np.array(lat) if lat else np.zeros(1)
    batches = server.stats()["batches"] - b0
    return {"frames": n, "frames_per_s": n / span, "p50_ms": float(np.percentile(arr, 50)),
            "p99_ms": float(np.percentile(arr, 99)), "mean_batch": n / max(batches, 1), "batches": batches,
            "offered_hz": rate_hz * len(frames_by_sensor)}
