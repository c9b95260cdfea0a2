/*
 * dc.h -- C-ABI of libdc, the GB300 (sm_103a) depth-completion library.
 *
 * The library runs the eight-step classical depth-completion chain of
 * Ku, Harakeh, Waslander, "In Defense of Classical Image Processing: Fast
 * Depth Completion on the CPU" (arXiv 1802.00036), Section IV:
 *
 *   1 invert valid depths, D_inv = 100 - D                    (Sec. IV-1)
 *   2 dilate with a 5x5 diamond (or another Fig. 4 element)   (Sec. IV-2)
 *   3 5x5 full-kernel morphological close                     (Sec. IV-3)
 *   4 7x7 full dilation written into empty pixels only        (Sec. IV-4)
 *   5 copy each column's topmost value up to row 0            (Sec. IV-5)
 *   6 31x31 full dilation written into empty pixels only      (Sec. IV-6)
 *   7 5x5 median, then 5x5 Gaussian (or bilateral) blur       (Sec. IV-7)
 *   8 invert back, D_out = 100 - D_inv                         (Sec. IV-8)
 *
 * It is the problem of Section III: a sparse M x N depth map in, a dense map
 * of the same size out; the colour image is not used.
 *
 * Conventions (all entry points):
 *   - Maps are row-major float32, 0 = empty, metres.  A pixel is empty when
 *     its value is below 0.1 (raw or inverted).  Row pitches are in
 *     elements, >= W.
 *   - Device pointers are CUDA device (or managed) memory of the context's
 *     device, owned by the caller; they must stay valid until the stream has
 *     passed the call.  Host pointers are ordinary or pinned host memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Device work is asynchronous on it unless stated.
 *   - Arguments are checked before any work is queued; a failed check
 *     queues nothing and returns DC_ERR_INVALID_ARG.  Asynchronous CUDA
 *     errors surface from dc_last_async_error() or from the next call.
 *   - A context is not thread-safe: use one per host thread.  Calls on one
 *     context run in call order on the device even when they name different
 *     streams (a later call's stream waits for the earlier call), because
 *     they share the context's scratch; use several contexts for overlap.
 *   - Results are deterministic: every pixel's arithmetic is independent of
 *     tiling, batch composition and launch shape.
 *   - Max and min ignore out-of-frame pixels; the median replicates the
 *     border; the blurs mirror it without repeating the edge (reflect-101).
 */
#ifndef DC_H
#define DC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DC_OK = 0,
    DC_ERR_INVALID_ARG = 1, /* bad pointer, size, pitch, aliasing or param  */
    DC_ERR_OOM = 2,         /* scratch would exceed the budget, or malloc   */
    DC_ERR_CUDA = 3,        /* a CUDA runtime call failed                   */
    DC_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up           */
    DC_ERR_UNSUPPORTED = 5  /* valid request this build cannot serve        */
} dc_status;

/* First structuring element, step 2 (Sec. IV-2, Fig. 4, Table 2). */
typedef enum {
    DC_K_DIAMOND5 = 0, /* |dy|+|dx| <= 2, 13 taps (paper's choice) */
    DC_K_FULL5 = 1,    /* 5x5                                      */
    DC_K_CROSS5 = 2,   /* dy == 0 or dx == 0 within 5x5, 9 taps    */
    DC_K_FULL3 = 3,    /* 3x3                                      */
    DC_K_CIRCLE5 = 4,  /* dy^2+dx^2 <= 5, 21 taps                  */
    DC_K_FULL7 = 5     /* 7x7                                      */
} dc_kernel;

/* Blur of step 7 after the optional median (Sec. IV-7, Table 3). */
typedef enum { DC_BLUR_NONE = 0, DC_BLUR_GAUSS = 1, DC_BLUR_BILATERAL = 2 } dc_blur;

/* Where the chain stops; every stop except DC_STOP_FULL returns the map in
 * the inverted domain (100 - depth on non-empty pixels, 0 elsewhere). */
typedef enum {
    DC_STOP_FULL = 0,
    DC_STOP_INVERT = 1,
    DC_STOP_DILATE = 2,
    DC_STOP_CLOSE = 3,
    DC_STOP_FILL7 = 4,
    DC_STOP_EXTEND = 5,
    DC_STOP_FILL_LARGE = 6,
    DC_STOP_MEDIAN = 7,
    DC_STOP_BLUR = 8
} dc_stage;

typedef struct {
    int first_kernel;  /* dc_kernel, step 2; paper: DC_K_DIAMOND5            */
    int large_fill;    /* odd side of the step-6 square, 3..63; paper: 31    */
    int median;        /* 1: 5x5 median in step 7; paper: 1                  */
    int blur;          /* dc_blur; paper: DC_BLUR_GAUSS                      */
    float sigma_space; /* bilateral spatial sigma in pixels (default 1.5)    */
    float sigma_color; /* bilateral range sigma, inverted metres (0.5)       */
    int extend_top;    /* 1: step 5 on (Sec. V-B skips 5 and 6 for clouds)   */
    int extend_rows;   /* < 0: extend to row 0; else at most this many rows  */
    int large_fill_on; /* 1: step 6 on                                       */
    int stop_after;    /* dc_stage                                           */
} dc_params;

/* One frame of a batch.  `in` and `out` are device pointers; they must not
 * overlap (every step reads a neighbourhood, so in-place is refused). */
typedef struct {
    const float* in;
    float* out;
    int H, W;
    int in_pitch, out_pitch; /* elements; >= W */
} dc_frame;

typedef struct dc_ctx dc_ctx;

/* Fill *p with the paper's final design (diamond 5x5, 31x31 fill, median +
 * Gaussian, full chain).  Returns DC_ERR_INVALID_ARG for p == NULL. */
dc_status dc_params_default(dc_params* p);

/* Create a context on CUDA device `device`.  The context owns its scratch
 * (the step-4 map between the two kernels, per-column top rows, frame
 * tables, staging for host calls).  Scratch grows on demand up to
 * `scratch_budget_bytes` (0 = no limit); a call that would need more
 * returns DC_ERR_OOM.  *ctx is set only on DC_OK. */
dc_status dc_create(dc_ctx** ctx, int device, size_t scratch_budget_bytes);

/* Run the chain on `n_frames` frames of any sizes, in one pass of the two
 * kernels over all frames' tiles.  Asynchronous on `stream`.  n_frames == 0
 * is a no-op.  Scratch grows (synchronously, outside any stream capture) if
 * this batch needs more than earlier ones. */
dc_status dc_complete(dc_ctx* ctx, const dc_frame* frames, int n_frames,
                      const dc_params* params, void* stream);

/* Same chain on `n` packed frames of one size: frame i is at
 * in + i*H*W and out + i*H*W (pitch W).  Device pointers; asynchronous. */
dc_status dc_complete_uniform(dc_ctx* ctx, const float* in, float* out, int n,
                              int H, int W, const dc_params* params, void* stream);

/* Same as dc_complete_uniform but `host_in` / `host_out` are HOST buffers
 * (pinned memory gives full copy bandwidth).  The batch is split into
 * chunks whose copy in, kernels and copy out overlap, on three streams of
 * the context (copy in, kernels, copy out); the copy in follows earlier
 * work on `stream`.  Returns when the result is in host_out. */
dc_status dc_complete_host(dc_ctx* ctx, const float* host_in, float* host_out, int n,
                           int H, int W, const dc_params* params, void* stream);

/* dc_complete_host without the final wait, for a stream of batches: the
 * call only enqueues its copies and kernels and returns, so that this
 * call's copy in runs while the previous call's copy out does (the context
 * stages through two buffer sets, used by turns).  host_in must stay
 * unchanged and host_out untouched until dc_host_wait(ctx) returns.  Work
 * enqueued later on `stream` is not ordered after this call (its kernels
 * run on a stream of the context, so that the next call's copy in need not
 * wait for them); a later call on this context, on any stream, is.  Errors
 * as dc_complete_host. */
dc_status dc_complete_host_async(dc_ctx* ctx, const float* host_in, float* host_out, int n,
                                 int H, int W, const dc_params* params, void* stream);

/* Wait until every copy out of earlier dc_complete_host_async calls on this
 * context has landed in host memory. */
dc_status dc_host_wait(dc_ctx* ctx);

/* Grow scratch now for batches of up to `n_frames` frames of up to H x W,
 * so that later calls of that size do not allocate. */
dc_status dc_reserve(dc_ctx* ctx, int n_frames, int H, int W);

/* LIDAR points to a sparse depth map, the step before the chain (Section
 * V: the benchmark projects the scans into the image with the camera
 * calibration).  Point i is (xyz[3i], xyz[3i+1], xyz[3i+2]) (device floats,
 * metres); P is a HOST array of 12 doubles, the row-major 3 x 4 projection.
 * (u, v, w) = P (x, y, z, 1) is evaluated in double in that order; a point
 * with w > 0 and d_min <= w <= d_max lands in pixel (floor(v/w), floor(u/w))
 * if inside H x W.  Each pixel of `depth` (device, row pitch `pitch`
 * floats) receives the smallest depth (float of w) of its points, others 0.
 * Asynchronous on `stream`. */
dc_status dc_project(dc_ctx* ctx, const float* xyz, long long n_points, const double* P, int H, int W,
                     double d_min, double d_max, float* depth, int pitch, void* stream);

/* Accuracy of n completed depth maps against ground truth: the KITTI
 * depth-completion measures the paper reports (Section V, Tables 1-3).  Over
 * pixels whose ground truth is valid (>= 0.1 m), per frame i:
 *   out[5i+0] RMSE (mm), out[5i+1] MAE (mm), out[5i+2] iRMSE (1/km),
 *   out[5i+3] iMAE (1/km), out[5i+4] number of valid pixels;
 * the inverse of an empty prediction (< 0.1) is taken as 0; all four
 * measures are 0 for a frame without valid pixels.  `pred` and `gt` are
 * device arrays of n packed H x W maps (metres); `out` is a HOST array of
 * 5 n doubles.  Sums per thread in float over 32 pixels, then in double.
 * Synchronous: returns when `out` is filled. */
dc_status dc_metrics(dc_ctx* ctx, const float* pred, const float* gt, int n, int H, int W,
                     double* out, void* stream);

/* Launch-shape choices of a context (never the results: every pixel's
 * arithmetic is the same under any tuning).  a_warps_per_sm: stage A (steps
 * 1-4) splits frames into row bands so that about this many warps per SM
 * run (more bands = more parallelism but more halo rows recomputed; 1..64,
 * default 8).  b_ctas_per_sm: persistent CTAs per SM of stage B (steps 5-8;
 * 1..5, default 5).  b_sparse_fill: a stage-B tile with at most this many
 * empty pixels near it fills them itself (step 6); a
 * tile with more goes to a second kernel that works on the whole window
 * region (0..160, default 160).  a_strip_cols: the width of stage A's column
 * strips, 128 (four columns per lane; least halo, for large batches) or 64
 * (two; twice the strips and half the work per warp, for one or a few
 * frames, where each warp's latency sets the time; default 128). */
typedef struct {
    int a_warps_per_sm;
    int b_ctas_per_sm;
    int b_sparse_fill;
    int a_strip_cols;
} dc_tuning;

dc_status dc_set_tuning(dc_ctx* ctx, const dc_tuning* t);
dc_status dc_get_tuning(const dc_ctx* ctx, dc_tuning* t);

/* Tunings per frame size, for calls that mix sizes.  A frame of H x W with
 * a recorded tuning takes its step-6 threshold (b_sparse_fill, the one
 * choice that is made per tile) from it in every call; the other knobs are
 * launch-wide and come from the context's tuning.  dc_autotune records its
 * choice for its H x W; this records t for H x W, replacing an earlier one,
 * or with t = NULL forgets every size.  At most DC_MAX_CLASS_TUNINGS sizes
 * (DC_ERR_UNSUPPORTED beyond); t is checked as by dc_set_tuning.  Drops the
 * context's cached CUDA graphs (they hold the old thresholds). */
#define DC_MAX_CLASS_TUNINGS 16
dc_status dc_set_class_tuning(dc_ctx* ctx, int H, int W, const dc_tuning* t);

/* Time dc_complete_uniform on the caller's n packed frames (device `in` /
 * `out`, as for dc_complete_uniform; `out` is overwritten) under a fixed set
 * of tunings (two rounds of one knob at a time), keep the fastest in the
 * context, record it for frames of H x W (as dc_set_class_tuning does; with
 * DC_MAX_CLASS_TUNINGS sizes recorded, the one recorded first makes room)
 * and return it in *best.  Synchronous; runs the chain ~170 times. */
dc_status dc_autotune(dc_ctx* ctx, const float* in, float* out, int n, int H, int W,
                      const dc_params* params, void* stream, dc_tuning* best);

/* Number of kernel launches the last dc_complete* call queued. */
int dc_last_launch_count(const dc_ctx* ctx);

/* Per-kernel timing.  With every >= 1, one later call in `every` (the
 * first, then each every-th) records CUDA events around each of its kernels
 * on the call's stream (a ring of the last DC_PROFILE_CALLS profiled calls);
 * 0 turns it off.  Each call restarts the ring.  An event between two
 * kernels keeps the second from being launched while the first finishes, so
 * profiling one call in several leaves the others' overlap intact.  Turning
 * it on allocates the events; every < 0 is DC_ERR_INVALID_ARG. */
#define DC_PROFILE_CALLS 4096
dc_status dc_set_profiling(dc_ctx* ctx, int every);

/* CUDA graphs for repeated calls (a stream of batches in the same buffers,
 * one launch for a whole batch).  With max_graphs >= 1, a dc_complete or
 * dc_complete_uniform call whose frames (pointers, sizes, pitches), params
 * and tuning equal those of a recent call is queued as one graph launch of
 * that call's kernels; another call runs as usual and is then captured, from
 * a stream of the context, into a graph kept among the max_graphs most
 * recently used.  The graphs read the frames' current contents: only the
 * pointers must match.  Results, ordering and errors are those of the call
 * without a graph; calls made while profiling is on are never captured, and
 * growing the scratch drops the graphs.  0 turns the cache off (the
 * default).  max_graphs outside 0..DC_MAX_GRAPHS is DC_ERR_INVALID_ARG.
 * Changing the size waits for the context's last call and drops the graphs. */
#define DC_MAX_GRAPHS 64
dc_status dc_set_graph_cache(dc_ctx* ctx, int max_graphs);

/* Number of graphs the context holds now (0 without a context). */
int dc_graph_cache_entries(const dc_ctx* ctx);

/* Wait for the profiled calls and write, for each of the last `max_calls`
 * profiled calls (oldest first), the milliseconds of stage A (steps 1-4)
 * and of stage B (steps 5-8; 0 when not launched) to ms[2*i], ms[2*i+1].
 * *n_out receives the number of calls written.  Clears the ring. */
dc_status dc_kernel_times(dc_ctx* ctx, float* ms, int max_calls, int* n_out);

/* First asynchronous error seen on the context's work so far (clears it).
 * Synchronises the context's last stream.  DC_ERR_TIMEOUT: a kernel's
 * bounded wait for its tensor copy of a region gave up (that kernel stopped;
 * its outputs are incomplete). */
dc_status dc_last_async_error(dc_ctx* ctx);

/* Testing hook: put the context in the state a failure would leave, without
 * any failure on the GPU, so that callers can test their error handling.
 *   DC_FAULT_WAIT: set the context's device error word, as stage B does when
 *     its bounded wait for a region copy gives up; the next
 *     dc_last_async_error() returns DC_ERR_TIMEOUT, the one after DC_OK.
 *   DC_FAULT_LAUNCH: the next call that launches kernels fails as if its
 *     first launch had been refused: it queues nothing and returns
 *     DC_ERR_CUDA, which dc_last_async_error() (or the call after) then
 *     reports once more, as for any CUDA error.
 * Returns DC_ERR_INVALID_ARG for a null context or an unknown fault. */
typedef enum { DC_FAULT_WAIT = 1, DC_FAULT_LAUNCH = 2 } dc_fault;
dc_status dc_inject_fault(dc_ctx* ctx, int fault);

/* Human-readable name of a status code (static storage). */
const char* dc_status_str(dc_status s);

/* Free the context and its scratch.  Waits for its queued work. */
void dc_destroy(dc_ctx* ctx);

/* ---- Allocation-free entry point (the paper has no counterpart) ----------
 *
 * For callers that must not allocate device memory at run time: code that
 * runs under a fixed memory plan (safety-certified or real-time stacks that
 * forbid cudaMalloc after start-up, because it can block, fragment memory or
 * fail unpredictably), plug-ins that only receive buffers from a host
 * framework, and allocators that forbid foreign allocations.  It takes no
 * context: the scratch it needs lives in one fixed array inside the library
 * (DC_NOALLOC_SCRATCH_BYTES of device memory that every GPU which loads the
 * library keeps until the process exits).
 *
 * Same chain and results as dc_complete_uniform on `n` packed frames of
 * H x W (device pointers, pitch W, `in` and `out` must not overlap),
 * asynchronous on `stream`.  Limits: n <= DC_NOALLOC_MAX_FRAMES,
 * n * H * roundup(W, 32) <= DC_NOALLOC_MAX_PIXELS and
 * n * roundup(W, 32) <= DC_NOALLOC_MAX_COLUMNS; larger requests return
 * DC_ERR_UNSUPPORTED and queue nothing (bad pointers, sizes, overlap or
 * params return DC_ERR_INVALID_ARG as elsewhere).  It calls no cudaMalloc, cudaFree or
 * other allocating routine; it only launches kernels.
 *
 * The first call on each device looks up the array's device address for that
 * device (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  Every call, on every stream, shares the one array and leaves the
 * last call's data in it; calls whose device work overlaps in time (other
 * streams, other host threads) race and give wrong results.  Order them on
 * one stream or with events. */
#define DC_NOALLOC_MAX_FRAMES 64
#define DC_NOALLOC_MAX_PIXELS (1 << 21)
#define DC_NOALLOC_MAX_COLUMNS 131072
#define DC_NOALLOC_WORK_INTS 65536 /* tile worklist; enough for any batch within the limits above */
#define DC_NOALLOC_SCRATCH_BYTES \
    (6 * DC_NOALLOC_MAX_PIXELS + 8 * DC_NOALLOC_MAX_COLUMNS + 4 * DC_NOALLOC_WORK_INTS + 65536)
dc_status dc_complete_noalloc(const float* in, float* out, int n, int H, int W,
                              const dc_params* params, void* stream);

/* ---- Serving: continuous batching on one GPU ----------------------------
 *
 * The paper has no counterpart: the chain served to several sensors whose
 * frames arrive one at a time (the serving workload: frames of mixed sizes
 * from several sensors, p50 / p99 latency beside throughput).  A worker
 * thread of the server owns all device work:
 *   - a submitted frame takes a free device slot (input and output frames of
 *     max_H x max_W; the slots share budget_bytes with the lanes' scratch)
 *     and is copied in; with no free slot it waits (back-pressure);
 *   - the copied frames form a batch when max_batch of them are ready or the
 *     oldest has waited deadline_us since it was submitted, and the batch
 *     runs as one dc_complete on a free lane (one of `lanes`, each with its
 *     own context, scratch reserved for a full batch, and stream), followed
 *     on that stream by the copies of the results into the callers' buffers;
 *   - once a lane's work has passed, its frames are reported done with their
 *     latency: from submission to the result in host memory.
 * Results are those of dc_complete for the frame alone.  Errors of the
 * worker's CUDA calls are sticky: returned by the next submit, poll or
 * stats call. */
typedef struct dc_server dc_server;

typedef struct {
    unsigned long long submitted; /* frames accepted by dc_server_submit */
    unsigned long long done;      /* frames whose result is in host memory */
    unsigned long long batches;   /* batches run */
    int slots;                    /* device slots (frames in flight at most) */
    int lanes;
} dc_server_stats;

/* Create a server on `device` for frames of at most max_H x max_W.
 * DC_ERR_OOM when budget_bytes cannot hold the lanes' scratch and one slot
 * (or device memory runs out); DC_ERR_INVALID_ARG for bad sizes, a negative
 * deadline, max_batch < 1 or lanes outside 1..16. */
dc_status dc_server_create(dc_server** srv, int device, int max_H, int max_W, size_t budget_bytes,
                           int deadline_us, int max_batch, int lanes, const dc_params* params);

/* Queue one H x W frame (host_in, float32 depths, row pitch W).  host_out
 * (H x W) receives the dense map; neither buffer may be touched until the
 * frame's tag comes back from dc_server_poll.  Pinned host memory keeps the
 * copies asynchronous.  Thread-safe.  DC_ERR_INVALID_ARG for null buffers or
 * a size beyond the server's maximum. */
dc_status dc_server_submit(dc_server* srv, const float* host_in, float* host_out, int H, int W,
                           unsigned long long tag);

/* The frames done since the last call, oldest first: up to `max` tags and
 * (when latency_ms is not null) their latencies in ms; *n_done receives the
 * count.  Thread-safe. */
dc_status dc_server_poll(dc_server* srv, unsigned long long* tags, double* latency_ms, int max,
                         int* n_done);

/* Counters of the server. */
dc_status dc_server_get_stats(dc_server* srv, dc_server_stats* stats);

/* Stop accepting frames, finish every queued one, free everything. */
void dc_server_destroy(dc_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* DC_H */
