"""Throughput of the depth-completion chain (arXiv 1802.00036, Section IV) on GB300.

Default workload: batched 352 x 1216 float32 sparse depth maps (64-beam,
~5% valid, depths 2-80 m), 64 frames per step, paper defaults (diamond 5x5,
31x31 fill, median + Gaussian).  A step is one dc_complete_uniform call over
the batch: both kernels, every step of the chain.  Inputs rotate over 4
resident batches (4 x 110 MB in, 4 x 110 MB out) so no step finds its data in
the 129 MB L2.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain C statement of the chain) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W = 352, 1216
BATCH = 64
ROTATE = 4
BYTES_PER_PX = 8            # algorithmic: read the sparse map once, write the dense map once
PROFILE_EVERY = 8           # steps per step with per-kernel CUDA events in the timed region
PAPER_CONTEXT = "paper: 90 Hz per frame on an Intel Core i7-7700K, Python + OpenCV (Sec. V-A)"
METRIC = "frames/s @352x1216 batched"


def workload_config(batch, blur):
    return {"workload": f"batched {batch} x 352x1216 float32 sparse depth maps, 64-beam ~5% valid, "
                        f"2-80 m; diamond5, fill31, median+{blur}",
            "batch": batch, "frame": "352x1216", "blur": blur}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--blur", default="gauss", choices=["gauss", "bilateral"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=1.5,
                    help="seconds of Poisson arrivals per rate in the serving leg (0: skip)")
    ap.add_argument("--quick", action="store_true",
                    help="timed batched steps only (no per-frame, e2e or CPU legs): for profiling")
    ap.add_argument("--tuning", default=None,
                    help="launch shape 'a_warps_per_sm,b_ctas_per_sm,b_sparse_fill[,a_strip_cols]' instead of the "
                         "tuning cache or the autotuner (e.g. 16,5,160: profile captures name it)")
    ap.add_argument("--params", default="",
                    help="chain parameters other than the paper's for the batched step, 'key=value,...' (e.g. "
                         "extend_rows=50: the capped extension of Sec. V-B), for profiling")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave the further workloads (configs 2-4) out of the bench line")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the bench line: one JSON line per further workload (the 375x1242 "
                         "batch with both blurs, the four-resolution mix, the element x fill-size sweep)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_counters(stage):
    """A stage's ncu counters per launch from the committed summary, or None
    if a source of the kernel changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            entry = json.load(fh)[stage]
        for path, digest in entry["sources"].items():
            with open(os.path.join(ROOT, path), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != digest:
                    return None
        return entry
    except Exception:
        return None


def measured_traffic(stage):
    """DRAM bytes per launch of a stage (ncu), or None."""
    entry = measured_counters(stage)
    if entry is None:
        return None
    return int(entry["dram_read_bytes"]) + int(entry["dram_write_bytes"])


# The ALU pipe (min/max, integer and logic operations) of one SM issues 2
# warp-instructions per clock (4 sub-partitions x 16 lanes); 152 SMs at 2070 MHz.
ALU_PEAK_G_WARP_INST = 152 * 2 * 2.070


def alu_roofline(stage, launch_ms):
    """The second bound: the kernel's ALU-pipe warp instructions per launch
    (ncu count of the same workload) over its CUDA-event launch time."""
    entry = measured_counters(stage)
    if entry is None or "alu_pipe_warp_insts" not in entry or not launch_ms:
        return None
    achieved = float(entry["alu_pipe_warp_insts"]) / (launch_ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": round(achieved, 1), "peak": round(ALU_PEAK_G_WARP_INST, 1),
            "unit": "G warp-instructions/s (ALU pipe)", "frac": round(achieved / ALU_PEAK_G_WARP_INST, 4),
            "basis": "executed ALU-pipe instructions per launch (ncu, profiles/traffic.json) over the "
                     "CUDA-event launch time; peak 152 SMs x 2 per clock x 2070 MHz"}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("DC_BENCH_GLOO") is None else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier_max(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def make_frames(n):
    from paper_1802_00036_gb300 import synth
    return synth.make_batch(n, synth.ONE_FRAME, config=0)


# ---------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, sampled every 20 ms (a
    timed region of a fraction of a second still gets several samples)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        if which == "start":
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((ts, float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 - 0.05 <= r[0] <= self.t1 + 0.05]
        note = "during timed region"
        if not inside and rows:
            inside = sorted(rows, key=lambda r: abs(r[0] - (self.t1 or r[0])))[:3]
            note = "nearest samples (timed region shorter than the sampling period)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside), "note": note}


# ------------------------------------------------------------------- CPU oracle

def oracle_throughput(frames, threads: int, rounds: int = 1):
    """Frames/s of the oracle over `frames`, one frame per thread at a time."""
    import concurrent.futures
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        for _ in range(rounds):
            list(ex.map(lambda f: oracle.complete(f), frames))
    dt = time.perf_counter() - t0
    return len(frames) * rounds / dt, dt


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(frames_pool):
    cores = os.cpu_count() or 1
    sample = [frames_pool[i % len(frames_pool)] for i in range(8 * cores)]
    fps, dt = oracle_throughput(sample, cores)
    one = [frames_pool[i % len(frames_pool)] for i in range(8)]
    fps1, dt1 = oracle_throughput(one, 1)
    return {"value": round(fps, 3), "unit": "frames/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{len(sample)} frames of 352x1216 (8 per core) through the single-threaded C oracle, "
                      f"one frame per thread on {cores} threads; {dt:.1f} s wall",
            "single_thread": {"value": round(fps1, 3), "unit": "frames/s",
                              "sample": f"{len(one)} frames on one thread; {dt1:.1f} s wall"},
            "context": PAPER_CONTEXT}


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step is a bounded sample of the
    workload (one frame per host core), frames/s over K timed steps."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = make_frames(min(cores, 16))
    step_frames = [pool[i % len(pool)] for i in range(cores)]
    for _ in range(args.warmup):
        oracle_throughput(step_frames, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_throughput(step_frames, cores)
    dt = time.perf_counter() - t0
    fps = cores * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": round(fps, 3), "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * dt / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(args.batch, args.blur),
                       sample=f"oracle on {cores} of the batch's frames per step, one per thread"),
        "cpu_baseline": {"value": round(fps, 3), "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{cores} frames per step, one per thread"},
        "e2e": {"value": round(fps, 3), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------- GPU

def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1802_00036_gb300 import dc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B = args.batch
    host = make_frames(B)                                     # (B, H, W) float32
    ins = [torch.from_numpy(host).to(dev) for _ in range(ROTATE)]
    outs = [torch.empty_like(ins[0]) for _ in range(ROTATE)]
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    ctx = dc.Context(local)
    extra = {}
    for item in (args.params.split(",") if args.params else []):
        k, v = item.split("=")
        extra[k.strip()] = int(v) if v.strip().lstrip("-").isdigit() else v.strip()
    p = dc.params(blur=args.blur, **extra)
    dc.dc_reserve(ctx.h, B, H, W)
    from paper_1802_00036_gb300 import tune
    if args.tuning:
        t = tuple(int(v) for v in args.tuning.split(","))
        dc.dc_set_tuning(ctx.h, *t)
        tuning = (dc.dc_get_tuning(ctx.h), "command line")
    else:
        tuning = tune.tuned(ctx, ins[0], outs[0], p, stream)  # before any timed region

    def step(i):
        dc.dc_complete_uniform(ctx.h, ins[i % ROTATE].data_ptr(), outs[i % ROTATE].data_ptr(), B, H, W, p, sp)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
    stream.synchronize()
    launches_per_step = dc.dc_last_launch_count(ctx.h)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # per-kernel events on one step in PROFILE_EVERY: an event between two
    # kernels keeps the second from launching while the first finishes
    dc.dc_set_profiling(ctx.h, PROFILE_EVERY)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    clocks.mark("start")
    ev0.record(stream)
    for i in range(args.steps):
        step(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("stop")
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ktimes = dc.dc_kernel_times(ctx.h)
    dc.dc_set_profiling(ctx.h, False)
    time.sleep(0.25)
    clocks.stop()
    ms_max = barrier_max(ms, world, dev)
    frames_total = B * args.steps * world
    fps = frames_total / (ms_max / 1e3)

    # per-kernel averages over the timed region
    a_ms = statistics.mean(k[0] for k in ktimes) if ktimes else None
    b_ms = statistics.mean(k[1] for k in ktimes) if ktimes else None

    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(fps, 1), "unit": "frames/s", "quick": True,
                              "params": extra, "kernels_ms": {"stage_a": a_ms, "stage_b": b_ms}}), flush=True)
        ctx.close()
        return

    # per-frame GPU form: one call per frame
    pf_steps = max(2, min(args.steps // 8, 50))
    with torch.cuda.stream(stream):
        for i in range(B):
            dc.dc_complete_uniform(ctx.h, ins[0][i].data_ptr(), outs[0][i].data_ptr(), 1, H, W, p, sp)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(pf_steps):
        for i in range(B):
            dc.dc_complete_uniform(ctx.h, ins[s % ROTATE][i].data_ptr(), outs[s % ROTATE][i].data_ptr(),
                                   1, H, W, p, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    pf_fps = B * pf_steps / (e0.elapsed_time(e1) / 1e3)

    # the batched step replayed from CUDA graphs (dc_set_graph_cache): one graph
    # per input set, captured on its first call
    dc.dc_set_graph_cache(ctx.h, ROTATE)
    for i in range(2 * ROTATE):
        step(i)
    stream.synchronize()
    g_steps = max(20, min(args.steps // 2, 200))
    e0.record(stream)
    for i in range(g_steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / g_steps
    g_graphs = dc.dc_graph_cache_entries(ctx.h)
    dc.dc_set_graph_cache(ctx.h, 0)

    # end to end through the host-buffer entry points (pinned), copies inside the timed region:
    # a stream of batches (each call's copy in overlaps the previous call's copy out; one wait
    # at the end), and one synchronous call per batch
    hins = [torch.from_numpy(host).pin_memory(), torch.from_numpy(host).pin_memory()]
    houts = [torch.empty_like(hins[0]).pin_memory() for _ in range(2)]
    hin, hout = hins[0], houts[0]
    e2e_steps = max(3, min(args.steps // 4, 100))
    for i in range(2):
        dc.dc_complete_host_async(ctx.h, hins[i % 2].data_ptr(), houts[i % 2].data_ptr(), B, H, W, p, sp)
    dc.dc_host_wait(ctx.h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        dc.dc_complete_host_async(ctx.h, hins[i % 2].data_ptr(), houts[i % 2].data_ptr(), B, H, W, p, sp)
    dc.dc_host_wait(ctx.h)
    stream.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = barrier_max(e2e_s, world, dev)
    e2e_fps = B * e2e_steps * world / e2e_s
    for _ in range(2):
        dc.dc_complete_host(ctx.h, hin.data_ptr(), hout.data_ptr(), B, H, W, p, sp)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dc.dc_complete_host(ctx.h, hin.data_ptr(), hout.data_ptr(), B, H, W, p, sp)
    e2e_sync_s = barrier_max(time.perf_counter() - t0, world, dev)
    e2e_sync_fps = B * e2e_steps * world / e2e_sync_s

    next_rows = run_next_rows(ctx, ins, outs, stream, B)
    configs = None if args.no_configs else run_configs(args, ctx)

    serving = None
    if args.serve_seconds > 0:
        serving = run_serving(args.serve_seconds)

    if rank != 0:
        ctx.close()
        return

    hbm, peak_kind = peaks()
    px = H * W
    # dominant kernel: its algorithmic bytes are its own input map read once and
    # output map written once (8 B per pixel), over its CUDA-event duration
    dom = "stage_b" if (b_ms or 0) >= (a_ms or 0) else "stage_a"
    dom_ms = max(a_ms or 0, b_ms or 0)
    achieved = BYTES_PER_PX * px * B / (dom_ms / 1e3) / 1e9 if dom_ms else None
    line = {
        "metric": METRIC, "value": round(fps, 1), "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(B, args.blur), params=extra or None,
                       parallelism="replicas" if world > 1 else "single",
                       tuning={"a_warps_per_sm": tuning[0][0], "b_ctas_per_sm": tuning[0][1],
                               "b_sparse_fill": tuning[0][2], "a_strip_cols": tuning[0][3], "source": tuning[1]},
                       l2=f"inputs rotate over {ROTATE} resident batches "
                          f"({ROTATE * B * px * 4 / 1e6:.0f} MB in + same out > 129 MB L2)"),
        "roofline": {
            "bound": "hbm", "kernel": dom,
            "achieved": round(achieved, 1) if achieved else None,
            "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4) if achieved else None,
            "peak_kind": peak_kind,
            "traffic": measured_traffic(dom) if B == BATCH else None,
            "traffic_unit": "bytes per launch (ncu, profiles/traffic.json)",
            "bytes_per_px": BYTES_PER_PX,
            "path_achieved": round(BYTES_PER_PX * px * fps / 1e9, 1),
            "path_frac": round(BYTES_PER_PX * px * fps / 1e9 / hbm, 4),
            "alu": alu_roofline(dom, dom_ms) if B == BATCH else None,
            # both kernels: the ALU bound and the DRAM traffic per launch (ncu)
            "by_kernel": {k: {"ms": round(k_ms, 4) if k_ms else None,
                              "alu": alu_roofline(k, k_ms) if B == BATCH else None,
                              "traffic": measured_traffic(k) if B == BATCH else None}
                          for k, k_ms in (("stage_a", a_ms), ("stage_b", b_ms))},
        },
        "kernels_ms": {"stage_a": round(a_ms, 4) if a_ms else None, "stage_b": round(b_ms, 4) if b_ms else None,
                       "calls_timed": len(ktimes), "profiled_every": PROFILE_EVERY},
        "per_frame": {"value": round(pf_fps, 1), "unit": "frames/s", "note": "one dc_complete call per frame"},
        "graph": {"value": round(B / g_ms * 1e3, 1), "unit": "frames/s", "ms_per_step": round(g_ms, 4),
                  "graphs": g_graphs, "note": "the batched step replayed from CUDA graphs (dc_set_graph_cache)"},
        "e2e": {"value": round(e2e_fps, 1), "unit": "frames/s",
                "h2d_bytes_per_step": int(hin.numel() * 4), "d2h_bytes_per_step": int(hout.numel() * 4),
                "note": "dc_complete_host_async on pinned host buffers, one batch per call, every copy in "
                        "the timed region (one dc_host_wait at its end)",
                "sync_call": {"value": round(e2e_sync_fps, 1), "unit": "frames/s",
                              "note": "dc_complete_host, returning when the batch is in host memory"}},
        "gpu_launches": launches_per_step * args.steps,
        "served": serving,
        "next_rows": next_rows,
        "configs": configs,
        "clocks": clocks.summary(),
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(host)
    elif not args.no_cpu_baseline and rank == 0:
        line["cpu_baseline"] = None
    ctx.close()
    print(json.dumps(line), flush=True)


def run_next_rows(ctx, ins, outs, stream, B):
    """The steps around the chain: accuracy measures of a completed batch
    against ground truth (8 B/px read) and LIDAR-to-image projection
    (12 B/point read, 4 B/px written), timed with CUDA events."""
    import numpy as np
    import torch

    from paper_1802_00036_gb300 import dc, synth
    hbm, _ = peaks()
    sp = stream.cuda_stream
    res = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # accuracy measures over the batch (outputs against inputs: only the time matters here)
    for _ in range(3):
        dc.dc_metrics(ctx.h, outs[0].data_ptr(), ins[1].data_ptr(), B, H, W, sp)
    reps = 20
    ev0.record(stream)
    for _ in range(reps):
        dc.dc_metrics(ctx.h, outs[0].data_ptr(), ins[1].data_ptr(), B, H, W, sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    gbs = 8.0 * B * H * W / (ms / 1e3) / 1e9
    res["metrics"] = {"frames_per_s": round(B / (ms / 1e3), 1), "ms_per_batch": round(ms, 4),
                      "achieved_GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                      "note": "includes the synchronous copy of the results to the host"}
    # the point-cloud mode of Section V-B (steps 5 and 6 off), on the batch, inputs rotating as in the
    # main timed loop; and with the extension capped at 50 rows and the large fill kept
    for name, kw in (("point_cloud_mode", dict(extend_top=False, large_fill_on=False)),
                     ("extend_capped_50", dict(extend_rows=50))):
        pm = dc.params(**kw)
        for i in range(4):
            dc.dc_complete_uniform(ctx.h, ins[i % len(ins)].data_ptr(), outs[i % len(outs)].data_ptr(), B, H, W, pm, sp)
        reps = 50
        ev0.record(stream)
        for i in range(reps):
            dc.dc_complete_uniform(ctx.h, ins[i % len(ins)].data_ptr(), outs[i % len(outs)].data_ptr(), B, H, W, pm, sp)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        gbs = BYTES_PER_PX * B * H * W / (ms / 1e3) / 1e9
        res[name] = {"frames_per_s": round(B / (ms / 1e3), 1), "ms_per_batch": round(ms, 4),
                     "achieved_GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
    # projection of one frame's point cloud (its returns lifted to 3D + 50k stray points)
    pts = synth.point_cloud(synth.ONE_FRAME, 4242, extra=50000)
    dpts = torch.from_numpy(pts).cuda()
    depth = torch.empty((H, W), device=outs[0].device)
    P = synth.camera_matrix(synth.ONE_FRAME).ravel()
    for _ in range(3):
        dc.dc_project(ctx.h, dpts.data_ptr(), len(pts), P, H, W, 0.1, 1e4, depth.data_ptr(), W, sp)
    reps = 200
    ev0.record(stream)
    for _ in range(reps):
        dc.dc_project(ctx.h, dpts.data_ptr(), len(pts), P, H, W, 0.1, 1e4, depth.data_ptr(), W, sp)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    gbs = (12.0 * len(pts) + 4.0 * H * W) / (ms / 1e3) / 1e9
    res["project"] = {"points": len(pts), "frames_per_s": round(1.0 / (ms / 1e3), 1),
                      "points_per_s": round(len(pts) / (ms / 1e3), 1), "ms_per_frame": round(ms, 5),
                      "achieved_GBps": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
    return res


def run_serving(seconds):
    """The continuous-batching server against one request per launch, on 8
    simulated sensors (Poisson arrivals) mixing 352x1216 and 512x2048 frames
    at 3-10 % density, device budget 2 GB, 2 ms batch deadline."""
    import torch

    from paper_1802_00036_gb300 import synth
    from paper_1802_00036_gb300.serve import NativeServer, drive_native
    sensors = 8
    pools = []
    for s in range(sensors):
        spec = synth.FrameSpec(352, 1216, 64, 0.05) if s % 2 == 0 else synth.FrameSpec(512, 2048, 128, 0.08)
        pool = []
        for k in range(3):
            dens = 0.03 + 0.07 * ((s * 3 + k) % 8) / 7.0
            f = synth.make_frame(synth.FrameSpec(spec.H, spec.W, spec.beams, dens), 5000 + 10 * s + k)
            pool.append(torch.from_numpy(f).pin_memory())
        pools.append(pool)
    out = {"sensors": sensors, "mix": "50/50 352x1216 / 512x2048, 3-10 % valid", "budget_bytes": 2 << 30,
           "deadline_ms": 2.0, "seconds_per_rate": seconds,
           "server": "dc_server (native worker): batches of up to 64 on 2 lanes; one frame per launch on 3 lanes",
           "client": "results into a ring of 256 pinned buffers (32 per sensor)",
           "latency": "scheduled arrival to result in pinned host memory", "rates": []}
    for rate in (10.0, 125.0, 1000.0, 4000.0, 8000.0):
        row = {"per_sensor_hz": rate}
        for name, kw in (("batched", dict(deadline_ms=2.0, max_batch=64, lanes=2)),
                         ("per_frame", dict(deadline_ms=0.0, max_batch=1, lanes=3))):
            srv = NativeServer(max_hw=(512, 2048), budget_bytes=2 << 30, **kw)
            try:
                drive_native(srv, pools, 1000.0, 0.3, seed=1, outstanding=256)        # warm-up: every lane
                res = drive_native(srv, pools, rate, seconds, seed=2, outstanding=256)
            finally:
                srv.close()
            row[name] = {k: round(v, 3) if isinstance(v, float) else v for k, v in res.items()}
        out["rates"].append(row)
    return out


def run_configs(args, ctx=None):
    """Throughput of the further workloads (configs 2-4 of the benchmark
    plan): a dict per workload.  Every timing: CUDA events around `steps`
    calls after `warmup` on rotating input sets whose total exceeds the L2;
    frames/s and algorithmic GB/s (8 B/px).  Clocks are sampled throughout."""
    import torch

    from paper_1802_00036_gb300 import dc, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    own = ctx is None
    if own:
        ctx = dc.Context(dev.index)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    steps, warm = max(min(args.steps // 10, 100), 20), max(args.warmup, 3)
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.2)
    clocks.mark("start")

    def timed(call, sets, n_steps=steps):
        for i in range(warm):
            call(i % sets)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(n_steps):
            call(i % sets)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n_steps  # ms per call

    def batch_sets(host, sets):
        return [torch.from_numpy(host).to(dev) for _ in range(sets)], [torch.empty(host.shape, device=dev)
                                                                        for _ in range(sets)]

    res = {}
    # the 64-frame 375x1242 batch, 4-6 % per frame: one call vs 64 calls, both blurs
    host = synth.make_batch(64, synth.UNIFORM_375, config=2, density_range=(0.04, 0.06))
    ins, outs = batch_sets(host, 4)
    n, H, W = host.shape
    rows = {}
    for blur in ("gauss", "bilateral"):
        p = dc.params(blur=blur)
        ms = timed(lambda i: dc.dc_complete_uniform(ctx.h, ins[i].data_ptr(), outs[i].data_ptr(), n, H, W, p, sp), 4)
        pf_steps = max(steps // 4, 5)
        ms1 = timed(lambda i: [dc.dc_complete_uniform(ctx.h, ins[i][k].data_ptr(), outs[i][k].data_ptr(), 1, H, W,
                                                      p, sp) for k in range(n)], 4, pf_steps)
        # the same from CUDA graphs (dc_set_graph_cache): the batch as one graph
        # launch per call; the 64 per-frame calls of one buffer set as 64 graphs
        dc.dc_set_graph_cache(ctx.h, 4)
        msg = timed(lambda i: dc.dc_complete_uniform(ctx.h, ins[i].data_ptr(), outs[i].data_ptr(), n, H, W, p, sp),
                    4)
        dc.dc_set_graph_cache(ctx.h, 64)
        msg1 = timed(lambda i: [dc.dc_complete_uniform(ctx.h, ins[0][k].data_ptr(), outs[0][k].data_ptr(), 1, H, W,
                                                       p, sp) for k in range(n)], 1, pf_steps)
        dc.dc_set_graph_cache(ctx.h, 0)
        rows[blur] = {"batched_frames_per_s": round(n / ms * 1e3, 1),
                      "per_frame_frames_per_s": round(n / ms1 * 1e3, 1),
                      "batched_graph_frames_per_s": round(n / msg * 1e3, 1),
                      "per_frame_graph_frames_per_s": round(n / msg1 * 1e3, 1),
                      "batched_GBps": round(n * H * W * 8 / ms / 1e6, 1)}
    res["batched_375x1242"] = {"workload": "64 x 375x1242, 4-6 % valid, 1-90 m, median + Gaussian / bilateral",
                               **rows}
    del ins, outs

    # the four-resolution mix: 32 frames of each, one call (dc_complete) and per resolution
    mix = []
    for k, spec in enumerate(synth.MIX):
        mix.append(synth.make_batch(32, spec, config=3, first=100 * k))
    dev_in = [[torch.from_numpy(b).to(dev) for b in mix] for _ in range(2)]
    dev_out = [[torch.empty(b.shape, device=dev) for b in mix] for _ in range(2)]
    p = dc.params()

    def frames_of(i):
        fr = []
        for b_in, b_out in zip(dev_in[i], dev_out[i]):
            _, h, w = b_in.shape
            fr += [(b_in[j].data_ptr(), b_out[j].data_ptr(), h, w, w, w) for j in range(b_in.shape[0])]
        return fr
    tables = [frames_of(0), frames_of(1)]
    ms = timed(lambda i: dc.dc_complete(ctx.h, tables[i], p, sp), 2)
    px = sum(b.size for b in mix)
    per_res = {}
    for k, b in enumerate(mix):
        _, h, w = b.shape
        msr = timed(lambda i: dc.dc_complete_uniform(ctx.h, dev_in[i][k].data_ptr(), dev_out[i][k].data_ptr(), 32, h,
                                                     w, p, sp), 2)
        per_res[f"{h}x{w}"] = round(32 / msr * 1e3, 1)
    # each resolution class with its own tuning (the autotuner's choice for a
    # batch of 32 of it, cached per GPU, batch, frame size and parameters);
    # the context's tuning is restored afterwards
    from paper_1802_00036_gb300 import tune
    keep = dc.dc_get_tuning(ctx.h)
    per_res_tuned = {}
    for k, b in enumerate(mix):
        _, h, w = b.shape
        choice, source = tune.tuned(ctx, dev_in[0][k], dev_out[0][k], p, stream)
        msr = timed(lambda i: dc.dc_complete_uniform(ctx.h, dev_in[i][k].data_ptr(), dev_out[i][k].data_ptr(), 32, h,
                                                     w, p, sp), 2)
        per_res_tuned[f"{h}x{w}"] = {"tuning": {"a_warps_per_sm": choice[0], "b_ctas_per_sm": choice[1],
                                                "b_sparse_fill": choice[2], "a_strip_cols": choice[3],
                                                "source": source},
                                     "frames_per_s": round(32 / msr * 1e3, 1)}
    # the one call again, each size's frames with their own step-6 threshold
    # (the knob that is chosen per tile; the others are launch-wide)
    dc.dc_set_tuning(ctx.h, *keep)
    ms_cls = timed(lambda i: dc.dc_complete(ctx.h, tables[i], p, sp), 2)
    dc.dc_set_class_tuning(ctx.h, 0, 0, None)
    res["uneven_mix"] = {"workload": "128 frames, 32 each of 256x512@3%, 352x1216@5%, 375x1242@5%, 512x2048@10%",
                         "one_call_frames_per_s": round(128 / ms * 1e3, 1),
                         "one_call_GBps": round(px * 8 / ms / 1e6, 1),
                         "per_resolution_batch_of_32_frames_per_s": per_res,
                         "per_resolution_tuned": per_res_tuned,
                         "one_call_per_size_threshold_frames_per_s": round(128 / ms_cls * 1e3, 1),
                         "tuning": {"a_warps_per_sm": keep[0], "b_ctas_per_sm": keep[1], "b_sparse_fill": keep[2],
                                    "a_strip_cols": keep[3], "note": "the one call and the untuned rows"}}
    del dev_in, dev_out

    # first element x large-fill size on 32 x 352x1216
    host = synth.make_batch(32, synth.ONE_FRAME, config=4)
    ins, outs = batch_sets(host, 4)
    n, H, W = host.shape
    rows = []
    for shape in ("diamond5", "full5", "cross5", "full3", "circle5", "full7"):
        for fill in (15, 31, 51):
            p = dc.params(first_kernel=shape, large_fill=fill)
            ms = timed(lambda i: dc.dc_complete_uniform(ctx.h, ins[i].data_ptr(), outs[i].data_ptr(), n, H, W, p,
                                                        sp), 4)
            rows.append({"first": shape, "fill": fill, "frames_per_s": round(n / ms * 1e3, 1),
                         "GBps": round(n * H * W * 8 / ms / 1e6, 1)})
    res["shape_sweep"] = {"workload": "32 x 352x1216, 5 % valid: first element x large fill", "rows": rows}
    clocks.mark("stop")
    time.sleep(0.2)
    clocks.stop()
    res["clocks"] = clocks.summary()
    res["timing"] = (f"CUDA events, {steps} calls after {warm} warm-up ({max(steps // 4, 5)} rounds of 64 calls "
                     f"for per-frame), inputs rotating over sets larger than the L2")
    if own:
        ctx.close()
    return res


def main():
    args = parse()
    if args.configs:
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        for name, row in run_configs(args).items():
            print(json.dumps({"config": name, **row} if isinstance(row, dict) else {name: row}), flush=True)
        return
    if args.impl == "reference":
        # the CPU oracle needs no process group: rank 0 runs it, others exit
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup(args.gpus)
    run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
