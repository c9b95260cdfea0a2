// dc_api.cu -- the C-ABI of libdc (include/dc.h): argument checks, scratch,
// frame tables and the kernel launches of each call.
#include "../../include/dc.h"
#include "common.cuh"

#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

using namespace dcgb;

namespace dcgb {

bool params_ok(const dc_params* p)
{
    if (!p) return false;
    if (p->first_kernel < DC_K_DIAMOND5 || p->first_kernel > DC_K_FULL7) return false;
    if (p->large_fill_on && (p->large_fill < 1 || p->large_fill > kMaxLargeFill || (p->large_fill % 2) == 0))
        return false;
    if (p->blur < DC_BLUR_NONE || p->blur > DC_BLUR_BILATERAL) return false;
    if (p->blur == DC_BLUR_BILATERAL && (!(p->sigma_space > 0.0f) || !(p->sigma_color > 0.0f) ||
                                         !std::isfinite(p->sigma_space) || !std::isfinite(p->sigma_color)))
        return false;
    if (p->stop_after < DC_STOP_FULL || p->stop_after > DC_STOP_BLUR) return false;
    return true;
}

}  // namespace dcgb

// dc_complete_host splits a batch into at most this many chunks so that the
// copy in of chunk i + 1, the kernels of chunk i and the copy out of chunk
// i - 1 overlap.
constexpr int kIoChunksMax = 16;

struct dc_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;  // 0 = unlimited
    Tuning tune = kDefaultTuning;
    // scratch
    float* c = nullptr;       // step-4 values off the key grid, all frames
    size_t c_cap = 0;         // floats
    unsigned short* ck = nullptr;  // step-4 maps as keys, all frames (same layout as c)
    unsigned long long* top = nullptr;  // per-column tops (top_pack), all frames
    size_t top_cap = 0;                 // entries
    int* work = nullptr;      // counters of both stages, then the step-6 tile list
    size_t work_cap = 0;      // ints
    double* acc = nullptr;    // accuracy sums and results, 10 doubles per frame
    int acc_cap = 0;          // frames
    int* err = nullptr;          // set by a device-side wait that gave up (device int)
    // the tensor map of C's keys for batches of one shape, kept while the layout holds
    CUtensorMap cmap{};
    const void* cmap_base = nullptr;
    int cmap_W = 0, cmap_H = 0, cmap_n = 0, cmap_pitch = 0;
    FrameDesc* table = nullptr;  // frame descriptors of the current call (device)
    int frames_cap = 0;          // descriptors
    cudaEvent_t done = nullptr;  // recorded after each call's last kernel
    // graphs of recent calls (dc_set_graph_cache): the call they replay, the
    // executable, its launches and when it was last used
    struct CachedGraph {
        std::vector<dc_frame> frames;
        dc_params params;
        Tuning tune;
        cudaGraphExec_t exec;
        int launches;
        unsigned long long used;
    };
    std::vector<CachedGraph> graphs;
    // per frame size, a tuning whose step-6 threshold that size's frames
    // take in every call (dc_set_class_tuning, dc_autotune); off while the
    // autotuner measures
    struct ClassTune {
        int H, W;
        Tuning t;
    };
    std::vector<ClassTune> classes;
    bool classes_off = false;
    int graph_max = 0;
    unsigned long long graph_tick = 0;
    cudaStream_t s_cap = nullptr;  // stream the graphs are captured from
    unsigned long long calls = 0;
    // staging for host calls: copy streams and events of the chunk pipeline
    // two staging sets, used by turns, so that one call's copy in can run
    // while the previous call's copy out does; io_read[k] marks the end of
    // the last kernel reading io_in[k], io_drained[k] the end of the last
    // copy out of io_out[k].  The kernels of host calls run on s_run, so
    // that the caller's stream orders only the copy in: were they on it, the
    // next call's copy in would wait for them.  Calls on other streams are
    // ordered after them through `done` like any change of stream.
    float* io_in[2] = {};
    float* io_out[2] = {};
    size_t io_cap = 0;        // floats each
    cudaStream_t s_in = nullptr, s_out = nullptr, s_run = nullptr;
    cudaEvent_t io_ev[2 * kIoChunksMax] = {};
    cudaEvent_t io_read[2] = {}, io_drained[2] = {};
    bool io_used[2] = {};
    int io_next = 0;
    // bookkeeping
    cudaStream_t last_stream = nullptr;
    cudaEvent_t last_done = nullptr;  // event of the latest call, or null
    int last_launches = 0;
    dc_status sticky = DC_OK;
    bool fail_next_launch = false;  // dc_inject_fault(DC_FAULT_LAUNCH)
    // profiling ring: 3 events per call (before A, between, after B)
    bool profiling = false;
    int prof_every = 1;                 // profile one call in prof_every
    unsigned long long prof_tick = 0;   // calls since profiling was turned on
    cudaEvent_t* prof_ev = nullptr;
    int prof_next = 0;     // next ring entry
    int prof_count = 0;    // valid entries
    int prof_has_b[DC_PROFILE_CALLS] = {};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

// The step-4 map takes a key (2 bytes) and a float (4 bytes) per position.
size_t scratch_bytes(size_t c_floats, size_t top_ints, int frames, size_t io_floats, size_t work_ints)
{
    return c_floats * (sizeof(float) + sizeof(unsigned short)) + top_ints * sizeof(unsigned long long) +
           work_ints * sizeof(int) + (size_t)frames * sizeof(FrameDesc) + 4 * io_floats * sizeof(float);
}


bool overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + nb && b0 < a0 + na;
}

void drop_graphs(dc_ctx* ctx)
{
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

dc_status grow(dc_ctx* ctx, size_t c_floats, size_t top_ints, int frames, size_t io_floats,
               size_t work_ints = 0)
{
    const bool need = c_floats > ctx->c_cap || top_ints > ctx->top_cap || frames > ctx->frames_cap ||
                      io_floats > ctx->io_cap || work_ints > ctx->work_cap;
    if (!need) return DC_OK;
    const size_t nc = c_floats > ctx->c_cap ? c_floats : ctx->c_cap;
    const size_t nt = top_ints > ctx->top_cap ? top_ints : ctx->top_cap;
    const int nf = frames > ctx->frames_cap ? frames : ctx->frames_cap;
    const size_t ni = io_floats > ctx->io_cap ? io_floats : ctx->io_cap;
    const size_t nw = work_ints > ctx->work_cap ? work_ints : ctx->work_cap;
    if (ctx->budget && scratch_bytes(nc, nt, nf, ni, nw) > ctx->budget) return DC_ERR_OOM;
    // queued work may still use the old buffers
    if (cudaDeviceSynchronize() != cudaSuccess) return DC_ERR_CUDA;
    drop_graphs(ctx);  // they hold the scratch pointers
    if (nc > ctx->c_cap) {
        cudaFree(ctx->c);
        cudaFree(ctx->ck);
        ctx->c = nullptr;
        ctx->ck = nullptr;
        ctx->c_cap = 0;
        ctx->cmap_base = nullptr;
        if (cudaMalloc(&ctx->c, nc * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&ctx->ck, nc * sizeof(unsigned short)) != cudaSuccess) {
            cudaGetLastError();
            return DC_ERR_OOM;
        }
        ctx->c_cap = nc;
    }
    if (nt > ctx->top_cap) {
        cudaFree(ctx->top);
        ctx->top = nullptr;
        ctx->top_cap = 0;
        if (cudaMalloc(&ctx->top, nt * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            return DC_ERR_OOM;
        }
        ctx->top_cap = nt;
    }
    if (nw > ctx->work_cap) {
        cudaFree(ctx->work);
        ctx->work = nullptr;
        ctx->work_cap = 0;
        if (cudaMalloc(&ctx->work, nw * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return DC_ERR_OOM; }
        ctx->work_cap = nw;
    }
    if (nf > ctx->frames_cap) {
        cudaFree(ctx->table);
        ctx->table = nullptr;
        ctx->frames_cap = 0;
        if (cudaMalloc(&ctx->table, nf * sizeof(FrameDesc)) != cudaSuccess) { cudaGetLastError(); return DC_ERR_OOM; }
        ctx->frames_cap = nf;
    }
    if (ni > ctx->io_cap) {
        for (int k = 0; k < 2; ++k) {
            cudaFree(ctx->io_in[k]);
            cudaFree(ctx->io_out[k]);
            ctx->io_in[k] = ctx->io_out[k] = nullptr;
        }
        ctx->io_cap = 0;
        for (int k = 0; k < 2; ++k)
            if (cudaMalloc(&ctx->io_in[k], ni * sizeof(float)) != cudaSuccess ||
                cudaMalloc(&ctx->io_out[k], ni * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                return DC_ERR_OOM;
            }
        ctx->io_cap = ni;
    }
    return DC_OK;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// The frame descriptors reach the device as kernel parameters, K at a time,
// and a kernel stores them; the same launch resets the column tops and
// stage A's unit counter.  A
// host-to-device copy would queue on the copy engine behind whatever large
// transfers the caller has in flight (dc_complete_host's own copy-in of the
// next chunk), holding back the kernels of this call.
template <int K>
struct TableChunk {
    FrameDesc d[K];
};
static_assert(sizeof(TableChunk<352>) + 64 <= 32764, "kernel parameter space");

template <int K>
__global__ void table_put(const __grid_constant__ TableChunk<K> src, FrameDesc* __restrict__ dst, int n,
                          unsigned long long* __restrict__ top, size_t top_ints, int* __restrict__ counter,
                          int* __restrict__ ffill)
{
    allow_next_kernel();  // stage A may launch; it waits for this kernel's writes
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    if (counter && tid == 0) *counter = 0;
    if (ffill && tid == 0) *ffill = 0;
    for (size_t i = tid; i < (size_t)n; i += stride) dst[i] = src.d[i];
    if (top)
        for (size_t i = tid; i < top_ints; i += stride) top[i] = kNoTopPacked;
}

template <int K>
cudaError_t table_put_chunk(const FrameDesc* desc, int n, FrameDesc* dst, unsigned long long* top, size_t top_ints,
                            int* counter, int* ffill, int sms, cudaStream_t stream)
{
    TableChunk<K> c;
    std::memcpy(c.d, desc, (size_t)n * sizeof(FrameDesc));
    size_t blocks = (top_ints + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > (size_t)2 * sms) blocks = (size_t)2 * sms;
    table_put<K><<<(unsigned)blocks, 256, 0, stream>>>(c, dst, n, top, top_ints, counter, ffill);
    return cudaGetLastError();
}

cudaError_t preload_kernels()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, table_put<8>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, table_put<64>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, table_put<352>);
    if (e == cudaSuccess) e = preload_stage_a();
    if (e == cudaSuccess) e = preload_stage_a_keys();
    if (e == cudaSuccess) e = preload_stage_b();
    if (e == cudaSuccess) e = preload_metrics();
    if (e == cudaSuccess) e = preload_project();
    return e;
}

// Store n descriptors at dst (chunks of up to 352 per launch), reset
// top_ints column tops, zero *counter and *ffill (when not null); returns
// the number of launches through *launches.
cudaError_t put_table(const FrameDesc* desc, int n, FrameDesc* dst, unsigned long long* top, size_t top_ints,
                      int* counter, int* ffill, int sms, cudaStream_t stream, int* launches)
{
    *launches = 0;
    for (int i = 0; i < n; i += 352) {
        const int m = n - i < 352 ? n - i : 352;
        unsigned long long* t = i == 0 ? top : nullptr;
        const size_t ti = i == 0 ? top_ints : 0;
        int* z = i == 0 ? counter : nullptr;
        int* ff = i == 0 ? ffill : nullptr;
        cudaError_t e = m <= 8    ? table_put_chunk<8>(desc + i, m, dst + i, t, ti, z, ff, sms, stream)
                      : m <= 64   ? table_put_chunk<64>(desc + i, m, dst + i, t, ti, z, ff, sms, stream)
                                  : table_put_chunk<352>(desc + i, m, dst + i, t, ti, z, ff, sms, stream);
        if (e != cudaSuccess) return e;
        ++*launches;
    }
    return cudaSuccess;
}

// Scratch one frame needs: step-4 map rows padded to 32 floats, tops padded.
size_t frame_c_floats(int H, int W) { return round_up((size_t)W, 32) * (size_t)H; }
size_t frame_top_ints(int W) { return round_up((size_t)W, 32); }

// cuTensorMapEncodeTiled from the driver, looked up once (no link-time
// dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        cudaGetLastError();
    }
    return fn;
}

// The tensor map of n step-4 key maps of H x W (rows `pitch` keys apart,
// frames H pitch keys apart) at `base`, with the box of stage B's region
// (kKeyBoxW x kKeyBoxH keys); false if it cannot be made (then the regions
// come by cp.async).
bool c_tensor_map(dc_ctx* ctx, const unsigned short* base, int n, int H, int W, int pitch)
{
    if (ctx->cmap_base == base && ctx->cmap_n == n && ctx->cmap_H == H && ctx->cmap_W == W &&
        ctx->cmap_pitch == pitch)
        return true;
    ctx->cmap_base = nullptr;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    const size_t row_bytes = (size_t)pitch * sizeof(unsigned short);
    if (!enc || (reinterpret_cast<uintptr_t>(base) % 16) != 0 || row_bytes % 16 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    const cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)row_bytes * H};
    const cuuint32_t box[3] = {(cuuint32_t)kKeyBoxW, (cuuint32_t)kKeyBoxH, 1};
    const cuuint32_t estride[3] = {1, 1, 1};
    if (enc(&ctx->cmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<unsigned short*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    ctx->cmap_base = base;
    ctx->cmap_n = n;
    ctx->cmap_H = H;
    ctx->cmap_W = W;
    ctx->cmap_pitch = pitch;
    return true;
}

// Queue one call.  With `capture` the launches go into a stream capture:
// no wait on the previous call's event, no profiling, no bookkeeping (the
// replay of the graph does those).
dc_status run(dc_ctx* ctx, const dc_frame* frames, int n, const dc_params* p, cudaStream_t stream,
              bool capture = false)
{
    ctx->last_launches = 0;
    if (n == 0) return DC_OK;

    // layout of scratch, stage-A units (strip x band) and stage-B tiles
    std::vector<FrameDesc> desc((size_t)n);
    const bool need_b = (p->stop_after == DC_STOP_FULL || p->stop_after >= DC_STOP_EXTEND);
    // the key kernel (full chain) takes the tuned strip width; the float
    // kernel alone (a stop before step 5) its own 128 columns
    const int strip_cols = need_b ? ctx->tune.a_strip_cols : 128;
    long long total_strips = 0;
    for (int i = 0; i < n; ++i) total_strips += stage_a_strips(frames[i].W, p->first_kernel, strip_cols);
    size_t c_off = 0, top_off = 0;
    long long tiles_a = 0, tiles_b = 0;
    for (int i = 0; i < n; ++i) {
        const dc_frame& f = frames[i];
        FrameDesc& d = desc[(size_t)i];
        d.in = f.in;
        d.out = f.out;
        d.H = f.H;
        d.W = f.W;
        d.in_pitch = f.in_pitch;
        d.out_pitch = f.out_pitch;
        d.c_pitch = (int)round_up((size_t)f.W, 32);
        d.tiles_x_a = stage_a_strips(f.W, p->first_kernel, strip_cols);
        d.ow_a = stage_a_strip_width(p->first_kernel, strip_cols);
        d.band_a = stage_a_band_rows(f.H, total_strips, (long long)ctx->tune.a_warps_per_sm * ctx->sm_count);
        d.tiles_x_b = ceil_div(f.W, kTileBW);
        d.sparse_fill = ctx->tune.b_sparse_fill;
        if (!ctx->classes_off)
            for (const auto& c : ctx->classes)
                if (c.H == f.H && c.W == f.W) d.sparse_fill = c.t.b_sparse_fill;
        d.base_a = (int)tiles_a;
        d.base_b = (int)tiles_b;
        tiles_a += (long long)d.tiles_x_a * ceil_div(f.H, d.band_a);
        tiles_b += (long long)d.tiles_x_b * ceil_div(f.H, kTileBH);
        d.c = reinterpret_cast<float*>(c_off);  // offsets until scratch is known
        d.ck = reinterpret_cast<unsigned short*>(c_off);
        d.top = reinterpret_cast<unsigned long long*>(top_off);
        c_off += frame_c_floats(f.H, f.W);
        top_off += frame_top_ints(f.W);
    }
    if (tiles_a > INT32_MAX / 2 || tiles_b > INT32_MAX / 2) return DC_ERR_UNSUPPORTED;

    // work: three counters, the step-6 tile list, the float step-6 list (a
    // count and the tiles)
    const size_t ff_off = need_b ? (size_t)tiles_b + 3 : 3;
    dc_status s = grow(ctx, need_b ? c_off : 0, need_b ? top_off : 0, n, 0,
                       need_b ? ff_off + 1 + (size_t)tiles_b : 3);
    if (s != DC_OK) return s;
    for (auto& d : desc) {
        d.ck = need_b ? ctx->ck + reinterpret_cast<size_t>(d.ck) : nullptr;
        d.c = need_b ? ctx->c + reinterpret_cast<size_t>(d.c) : nullptr;
        d.top = need_b ? ctx->top + reinterpret_cast<size_t>(d.top) : nullptr;
    }

    if (ctx->fail_next_launch) {  // an injected launch failure: nothing is queued
        ctx->fail_next_launch = false;
        return DC_ERR_CUDA;
    }
    // calls share the scratch: order this one after the previous call
    if (!capture && ctx->last_done && stream != ctx->last_stream &&
        cudaStreamWaitEvent(stream, ctx->last_done, 0) != cudaSuccess)
        return DC_ERR_CUDA;
    // the descriptors and the reset of the tops, written by a kernel
    int table_launches = 0;
    int* ffill = need_b ? ctx->work + ff_off : nullptr;
    if (put_table(desc.data(), n, ctx->table, need_b ? ctx->top : nullptr, need_b ? top_off : 0, ctx->work + 2,
                  ffill, ctx->sm_count, stream, &table_launches) != cudaSuccess)
        return DC_ERR_CUDA;

    cudaEvent_t* ev = nullptr;
    if (!capture && ctx->profiling && ctx->prof_tick++ % (unsigned long long)ctx->prof_every == 0) {
        ev = ctx->prof_ev + 3 * ctx->prof_next;
        ctx->prof_has_b[ctx->prof_next] = need_b ? 1 : 0;
        ctx->prof_next = (ctx->prof_next + 1) % DC_PROFILE_CALLS;
        if (ctx->prof_count < DC_PROFILE_CALLS) ++ctx->prof_count;
        if (cudaEventRecord(ev[0], stream) != cudaSuccess) return DC_ERR_CUDA;
    }
    const int stop_a = need_b ? kStopFull : p->stop_after;
    bool one_shape = true;
    for (int i = 1; i < n && one_shape; ++i) one_shape = frames[i].H == frames[0].H && frames[i].W == frames[0].W;
    const int band_stride = one_shape ? (int)total_strips : 0;
    // the full chain: steps 1-4 on keys (a unit whose inputs are off the
    // key grid on floats, by the same warp); a stop before step 5: the float
    // kernel on every unit
    cudaError_t e = cudaSuccess;
    if (stop_a == kStopFull) {
        e = launch_stage_a_keys(ctx->table, n, (int)tiles_a, p->first_kernel, strip_cols, ctx->work, band_stride,
                                ctx->sm_count, stream);
    } else {
        e = launch_stage_a(ctx->table, n, (int)tiles_a, p->first_kernel, stop_a, ctx->work, band_stride,
                           ctx->sm_count, stream);
    }
    if (e != cudaSuccess) return DC_ERR_CUDA;
    ctx->last_launches = table_launches + 1;
    if (ev && cudaEventRecord(ev[1], stream) != cudaSuccess) return DC_ERR_CUDA;
    if (need_b) {
        StageBParams bp{};
        bp.large_fill_on = p->large_fill_on ? 1 : 0;
        bp.large_radius = p->large_fill_on ? p->large_fill / 2 : 0;
        bp.median = p->median ? 1 : 0;
        bp.blur = p->blur;
        bp.extend_top = p->extend_top ? 1 : 0;
        bp.extend_rows = p->extend_rows;
        bp.stop = p->stop_after;
        bp.row_stride = one_shape ? (int)(((frames[0].W + kTileBW - 1) / kTileBW) * (long long)n) : 0;
        const double ss = p->blur == DC_BLUR_BILATERAL ? p->sigma_space : 1.0;
        const double sc = p->blur == DC_BLUR_BILATERAL ? p->sigma_color : 1.0;
        for (int r2 = 0; r2 < 5; ++r2) bp.ws[r2] = (float)std::exp(-(double)r2 / (2.0 * ss * ss));
        bp.inv_2sc2 = (float)(1.0 / (2.0 * sc * sc));
        // frames of one shape: C's keys are one W x H x n array, one tensor map
        const bool tma = one_shape && c_tensor_map(ctx, desc[0].ck, n, frames[0].H, frames[0].W, desc[0].c_pitch);
        bp.tma = tma ? 1 : 0;
        e = launch_stage_b(ctx->table, n, (int)tiles_b, bp, ctx->work, ffill, ctx->sm_count, ctx->tune.b_ctas_per_sm,
                           tma ? &ctx->cmap : nullptr, ctx->err, stream);
        if (e != cudaSuccess) return DC_ERR_CUDA;
        // stage A is one kernel, stage B one plus the step-6 passes when step 6 can run
        ctx->last_launches = table_launches + 1 + stage_b_launches(bp);
    }
    if (ev && cudaEventRecord(ev[2], stream) != cudaSuccess) return DC_ERR_CUDA;
    if (capture) return DC_OK;
    if (cudaEventRecord(ctx->done, stream) != cudaSuccess) return DC_ERR_CUDA;
    ctx->last_done = ctx->done;
    ctx->last_stream = stream;
    ++ctx->calls;
    return DC_OK;
}

// run() through the graph cache.  A call equal to a recent one (frames,
// params, tuning) replays its graph; another runs as usual and is then
// captured, from the context's own stream, for the next time (scratch has
// grown by then, so the capture allocates nothing).  A capture that fails
// only leaves the call without a graph.
dc_status run_cached(dc_ctx* ctx, const dc_frame* frames, int n, const dc_params* p, cudaStream_t stream)
{
    if (ctx->graph_max <= 0 || ctx->profiling || n == 0) return run(ctx, frames, n, p, stream);
    for (auto& g : ctx->graphs) {
        if ((int)g.frames.size() != n || std::memcmp(&g.params, p, sizeof(dc_params)) != 0 ||
            std::memcmp(&g.tune, &ctx->tune, sizeof(Tuning)) != 0 ||
            std::memcmp(g.frames.data(), frames, sizeof(dc_frame) * (size_t)n) != 0)
            continue;
        if (ctx->last_done && stream != ctx->last_stream &&
            cudaStreamWaitEvent(stream, ctx->last_done, 0) != cudaSuccess)
            return DC_ERR_CUDA;
        if (cudaGraphLaunch(g.exec, stream) != cudaSuccess || cudaEventRecord(ctx->done, stream) != cudaSuccess)
            return DC_ERR_CUDA;
        ctx->last_done = ctx->done;
        ctx->last_stream = stream;
        ctx->last_launches = g.launches;
        ++ctx->calls;
        g.used = ++ctx->graph_tick;
        return DC_OK;
    }
    dc_status s = run(ctx, frames, n, p, stream);
    if (s != DC_OK) return s;
    const int launches = ctx->last_launches;
    if (!ctx->s_cap && cudaStreamCreateWithFlags(&ctx->s_cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return DC_OK;
    }
    if (cudaStreamBeginCapture(ctx->s_cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return DC_OK;
    }
    const dc_status cs = run(ctx, frames, n, p, ctx->s_cap, true);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->s_cap, &graph);
    cudaGraphExec_t exec = nullptr;
    const bool ok = cs == DC_OK && ce == cudaSuccess && graph &&
                    cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    ctx->last_launches = launches;
    if (!ok) {
        cudaGetLastError();
        return DC_OK;
    }
    if ((int)ctx->graphs.size() >= ctx->graph_max) {  // the least recently used makes room
        size_t lru = 0;
        for (size_t i = 1; i < ctx->graphs.size(); ++i)
            if (ctx->graphs[i].used < ctx->graphs[lru].used) lru = i;
        cudaGraphExecDestroy(ctx->graphs[lru].exec);
        ctx->graphs.erase(ctx->graphs.begin() + (long)lru);
    }
    ctx->graphs.push_back(dc_ctx::CachedGraph{std::vector<dc_frame>(frames, frames + n), *p, ctx->tune, exec,
                                              launches, ++ctx->graph_tick});
    return DC_OK;
}

dc_status check_frames(const dc_frame* frames, int n)
{
    if (n < 0 || (n > 0 && !frames)) return DC_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const dc_frame& f = frames[i];
        if (!f.in || !f.out || f.H < 1 || f.W < 1 || f.in_pitch < f.W || f.out_pitch < f.W)
            return DC_ERR_INVALID_ARG;
        if ((size_t)f.H * (size_t)f.in_pitch > (size_t)INT32_MAX * 4) return DC_ERR_UNSUPPORTED;
        if (((uintptr_t)f.in % sizeof(float)) != 0 || ((uintptr_t)f.out % sizeof(float)) != 0)
            return DC_ERR_INVALID_ARG;
        const size_t in_bytes = ((size_t)(f.H - 1) * f.in_pitch + f.W) * sizeof(float);
        const size_t out_bytes = ((size_t)(f.H - 1) * f.out_pitch + f.W) * sizeof(float);
        for (int j = 0; j < n; ++j) {
            const dc_frame& g = frames[j];
            const size_t g_in = ((size_t)(g.H - 1) * g.in_pitch + g.W) * sizeof(float);
            if (overlap(f.out, out_bytes, g.in, g_in)) return DC_ERR_INVALID_ARG;
            if (j != i) {
                const size_t g_out = ((size_t)(g.H - 1) * g.out_pitch + g.W) * sizeof(float);
                if (overlap(f.out, out_bytes, g.out, g_out)) return DC_ERR_INVALID_ARG;
            }
        }
        (void)in_bytes;
    }
    return DC_OK;
}

dc_status note(dc_ctx* ctx, dc_status s)
{
    if (s == DC_ERR_CUDA && ctx->sticky == DC_OK) ctx->sticky = s;
    return s;
}

}  // namespace

extern "C" {

dc_status dc_params_default(dc_params* p)
{
    if (!p) return DC_ERR_INVALID_ARG;
    p->first_kernel = DC_K_DIAMOND5;
    p->large_fill = 31;
    p->median = 1;
    p->blur = DC_BLUR_GAUSS;
    p->sigma_space = 1.5f;
    p->sigma_color = 0.5f;
    p->extend_top = 1;
    p->extend_rows = -1;
    p->large_fill_on = 1;
    p->stop_after = DC_STOP_FULL;
    return DC_OK;
}

dc_status dc_create(dc_ctx** out, int device, size_t scratch_budget_bytes)
{
    if (!out) return DC_ERR_INVALID_ARG;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) { cudaGetLastError(); return DC_ERR_CUDA; }
    if (device < 0 || device >= count) return DC_ERR_INVALID_ARG;
    dc_ctx* ctx = new (std::nothrow) dc_ctx();
    if (!ctx) return DC_ERR_OOM;
    ctx->device = device;
    ctx->budget = scratch_budget_bytes;
    DeviceGuard g(device);
    bool ok = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->done, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&ctx->err, sizeof(int)) == cudaSuccess && cudaMemset(ctx->err, 0, sizeof(int)) == cudaSuccess;
    // every kernel loaded now: no call pays CUDA's lazy module loading (tens
    // of milliseconds, at the first launch of each kernel otherwise)
    ok = ok && preload_kernels() == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dc_destroy(ctx);
        return DC_ERR_CUDA;
    }
    *out = ctx;
    return DC_OK;
}

dc_status dc_reserve(dc_ctx* ctx, int n_frames, int H, int W)
{
    if (!ctx || n_frames < 0 || H < 1 || W < 1) return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    const size_t tiles = (size_t)ceil_div(W, kTileBW) * (size_t)ceil_div(H, kTileBH) * (size_t)n_frames;
    // work: three counters, the step-6 list, the float step-6 list and its count
    return note(ctx, grow(ctx, frame_c_floats(H, W) * (size_t)n_frames,
                          frame_top_ints(W) * (size_t)n_frames, n_frames, 0, 2 * tiles + 4));
}

dc_status dc_complete(dc_ctx* ctx, const dc_frame* frames, int n_frames, const dc_params* params,
                      void* stream)
{
    if (!ctx || !params_ok(params)) return DC_ERR_INVALID_ARG;
    dc_status s = check_frames(frames, n_frames);
    if (s != DC_OK) return s;
    if (ctx->sticky != DC_OK) {
        s = ctx->sticky;
        ctx->sticky = DC_OK;
        return s;
    }
    DeviceGuard g(ctx->device);
    return note(ctx, run_cached(ctx, frames, n_frames, params, (cudaStream_t)stream));
}

dc_status dc_complete_uniform(dc_ctx* ctx, const float* in, float* out, int n, int H, int W,
                              const dc_params* params, void* stream)
{
    if (!ctx || n < 0 || (n > 0 && (!in || !out || H < 1 || W < 1))) return DC_ERR_INVALID_ARG;
    std::vector<dc_frame> fr((size_t)n);
    const size_t step = (size_t)H * (size_t)W;
    for (int i = 0; i < n; ++i) fr[(size_t)i] = dc_frame{in + i * step, out + i * step, H, W, W, W};
    // packed frames of one size: the overlap check reduces to the two spans
    if (n > 0 && overlap(in, step * n * sizeof(float), out, step * n * sizeof(float)))
        return DC_ERR_INVALID_ARG;
    if (!params_ok(params)) return DC_ERR_INVALID_ARG;
    if (ctx->sticky != DC_OK) {
        dc_status s = ctx->sticky;
        ctx->sticky = DC_OK;
        return s;
    }
    if (((uintptr_t)in % sizeof(float)) != 0 || ((uintptr_t)out % sizeof(float)) != 0)
        return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return note(ctx, run_cached(ctx, fr.data(), n, params, (cudaStream_t)stream));
}

namespace {

// Enqueue a host-buffer call: copy in, kernels and copy out of up to
// `chunks` chunks, through staging set ctx->io_next.  Nothing waits on the host.  The
// copies run on s_in and s_out, the kernels on s_run; `st` orders the copy in
// only.
dc_status host_enqueue(dc_ctx* ctx, const float* host_in, float* host_out, int n, int H, int W,
                       const dc_params* params, cudaStream_t st, int chunks)
{
    const size_t frame = (size_t)H * W;
    dc_status s = grow(ctx, 0, 0, 0, (size_t)n * frame);
    if (s != DC_OK) return note(ctx, s);
    if (!ctx->s_in) {
        bool ok = cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&ctx->s_run, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; ok && i < 2 * kIoChunksMax; ++i)
            ok = cudaEventCreateWithFlags(&ctx->io_ev[i], cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < 2; ++k)
            ok = cudaEventCreateWithFlags(&ctx->io_read[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&ctx->io_drained[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return note(ctx, DC_ERR_CUDA);
    }
    const int set = ctx->io_next;
    float* io_in = ctx->io_in[set];
    float* io_out = ctx->io_out[set];
    // chunks of at least 8 frames, so that each still fills the GPU.  A
    // single call overlaps its own copies and kernels through 4 chunks; a
    // stream of calls overlaps one call's kernels with the copies of its
    // neighbours, where 2 larger chunks do better (shorter kernels per frame,
    // fewer copy starts)
    int per = (n + chunks - 1) / chunks;
    if (per < 8) per = 8;
    if (per > n) per = n;
    // the copy in follows earlier work on `stream` (which may have produced
    // host_in) and the last kernel that read this staging set; the kernels
    // follow the last copy out of this set's output staging
    cudaStream_t ks = ctx->s_run;
    cudaEvent_t start = ctx->io_ev[0];
    if (cudaEventRecord(start, st) != cudaSuccess || cudaStreamWaitEvent(ctx->s_in, start, 0) != cudaSuccess ||
        (ctx->io_used[set] && (cudaStreamWaitEvent(ctx->s_in, ctx->io_read[set], 0) != cudaSuccess ||
                               cudaStreamWaitEvent(ks, ctx->io_drained[set], 0) != cudaSuccess)))
        return note(ctx, DC_ERR_CUDA);
    int k = 0;
    for (int f0 = 0; f0 < n; f0 += per, ++k) {
        const int m = (n - f0 < per) ? n - f0 : per;
        const size_t off = (size_t)f0 * frame, bytes = (size_t)m * frame * sizeof(float);
        cudaEvent_t in_done = ctx->io_ev[2 * k], run_done = ctx->io_ev[2 * k + 1];
        if (cudaMemcpyAsync(io_in + off, host_in + off, bytes, cudaMemcpyHostToDevice, ctx->s_in) != cudaSuccess ||
            cudaEventRecord(in_done, ctx->s_in) != cudaSuccess || cudaStreamWaitEvent(ks, in_done, 0) != cudaSuccess)
            return note(ctx, DC_ERR_CUDA);
        s = dc_complete_uniform(ctx, io_in + off, io_out + off, m, H, W, params, ks);
        if (s != DC_OK) return s;
        if (cudaEventRecord(run_done, ks) != cudaSuccess || cudaStreamWaitEvent(ctx->s_out, run_done, 0) != cudaSuccess ||
            cudaMemcpyAsync(host_out + off, io_out + off, bytes, cudaMemcpyDeviceToHost, ctx->s_out) != cudaSuccess)
            return note(ctx, DC_ERR_CUDA);
    }
    if (cudaEventRecord(ctx->io_read[set], ks) != cudaSuccess ||
        cudaEventRecord(ctx->io_drained[set], ctx->s_out) != cudaSuccess)
        return note(ctx, DC_ERR_CUDA);
    ctx->io_used[set] = true;
    ctx->io_next = set ^ 1;
    return DC_OK;
}

bool host_args_ok(const dc_ctx* ctx, const float* host_in, const float* host_out, int n, int H, int W,
                  const dc_params* params)
{
    return ctx && n >= 0 && (n == 0 || (host_in && host_out && H >= 1 && W >= 1)) && params_ok(params);
}

}  // namespace

dc_status dc_complete_host(dc_ctx* ctx, const float* host_in, float* host_out, int n, int H, int W,
                           const dc_params* params, void* stream)
{
    if (!host_args_ok(ctx, host_in, host_out, n, H, W, params)) return DC_ERR_INVALID_ARG;
    if (n == 0) return DC_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    dc_status s = host_enqueue(ctx, host_in, host_out, n, H, W, params, st, 4);
    if (s != DC_OK) return s;
    if (cudaStreamSynchronize(ctx->s_out) != cudaSuccess || cudaStreamSynchronize(ctx->s_run) != cudaSuccess)
        return note(ctx, DC_ERR_CUDA);
    return DC_OK;
}

dc_status dc_complete_host_async(dc_ctx* ctx, const float* host_in, float* host_out, int n, int H, int W,
                                 const dc_params* params, void* stream)
{
    if (!host_args_ok(ctx, host_in, host_out, n, H, W, params)) return DC_ERR_INVALID_ARG;
    if (n == 0) return DC_OK;
    DeviceGuard g(ctx->device);
    return host_enqueue(ctx, host_in, host_out, n, H, W, params, (cudaStream_t)stream, 2);
}

dc_status dc_host_wait(dc_ctx* ctx)
{
    if (!ctx) return DC_ERR_INVALID_ARG;
    if (!ctx->s_out) return DC_OK;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize(ctx->s_out) != cudaSuccess) return note(ctx, DC_ERR_CUDA);
    return DC_OK;
}

int dc_last_launch_count(const dc_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

dc_status dc_project(dc_ctx* ctx, const float* xyz, long long n_points, const double* P, int H, int W,
                     double d_min, double d_max, float* depth, int pitch, void* stream)
{
    if (!ctx || !P || !depth || n_points < 0 || (n_points > 0 && !xyz) || H < 1 || W < 1 || pitch < W ||
        !(d_min >= 0.0) || !(d_max >= d_min))
        return DC_ERR_INVALID_ARG;
    for (int k = 0; k < 12; ++k)
        if (!std::isfinite(P[k])) return DC_ERR_INVALID_ARG;
    if (((uintptr_t)depth % sizeof(float)) != 0 || ((uintptr_t)xyz % sizeof(float)) != 0) return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (launch_project(xyz, n_points, P, H, W, d_min, d_max, depth, pitch, st) != cudaSuccess)
        return note(ctx, DC_ERR_CUDA);
    ctx->last_launches = n_points > 0 ? 2 : 1;
    return DC_OK;
}

dc_status dc_metrics(dc_ctx* ctx, const float* pred, const float* gt, int n, int H, int W, double* out,
                     void* stream)
{
    if (!ctx || n < 0 || (n > 0 && (!pred || !gt || !out || H < 1 || W < 1))) return DC_ERR_INVALID_ARG;
    if (n == 0) return DC_OK;
    if (((uintptr_t)pred % sizeof(float)) != 0 || ((uintptr_t)gt % sizeof(float)) != 0) return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (n > ctx->acc_cap) {
        if (ctx->budget && (size_t)n * 10 * sizeof(double) > ctx->budget) return DC_ERR_OOM;
        if (cudaDeviceSynchronize() != cudaSuccess) return note(ctx, DC_ERR_CUDA);
        cudaFree(ctx->acc);
        ctx->acc = nullptr;
        ctx->acc_cap = 0;
        if (cudaMalloc(&ctx->acc, sizeof(double) * 10 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return DC_ERR_OOM;
        }
        ctx->acc_cap = n;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->last_done && st != ctx->last_stream && cudaStreamWaitEvent(st, ctx->last_done, 0) != cudaSuccess)
        return note(ctx, DC_ERR_CUDA);
    double* res = ctx->acc + 5 * (size_t)n;
    if (launch_metrics(pred, gt, n, H, W, ctx->acc, res, st) != cudaSuccess) return note(ctx, DC_ERR_CUDA);
    ctx->last_launches = 2;
    if (cudaMemcpyAsync(out, res, sizeof(double) * 5 * (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return note(ctx, DC_ERR_CUDA);
    return DC_OK;
}

namespace {
bool tuning_ok(const dc_tuning* t)
{
    return t && t->a_warps_per_sm >= 1 && t->a_warps_per_sm <= 64 && t->b_ctas_per_sm >= 1 &&
           t->b_ctas_per_sm <= 5 && t->b_sparse_fill >= 0 && t->b_sparse_fill <= 160 &&
           (t->a_strip_cols == 64 || t->a_strip_cols == 128);
}

// Record (or replace) the tuning of frames of H x W; cached graphs hold the
// old per-frame thresholds, so they go.  A full table refuses a new size,
// or with evict_oldest drops the size recorded first to make room.
dc_status put_class(dc_ctx* ctx, int H, int W, const Tuning& t, bool evict_oldest)
{
    for (auto& c : ctx->classes)
        if (c.H == H && c.W == W) {
            c.t = t;
            drop_graphs(ctx);
            return DC_OK;
        }
    if ((int)ctx->classes.size() >= DC_MAX_CLASS_TUNINGS) {
        if (!evict_oldest) return DC_ERR_UNSUPPORTED;
        ctx->classes.erase(ctx->classes.begin());
    }
    ctx->classes.push_back(dc_ctx::ClassTune{H, W, t});
    drop_graphs(ctx);
    return DC_OK;
}
}  // namespace

dc_status dc_set_tuning(dc_ctx* ctx, const dc_tuning* t)
{
    if (!ctx || !tuning_ok(t)) return DC_ERR_INVALID_ARG;
    ctx->tune = Tuning{t->a_warps_per_sm, t->b_ctas_per_sm, t->b_sparse_fill, t->a_strip_cols};
    return DC_OK;
}

dc_status dc_set_class_tuning(dc_ctx* ctx, int H, int W, const dc_tuning* t)
{
    if (!ctx) return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!t) {
        if (!ctx->classes.empty()) drop_graphs(ctx);
        ctx->classes.clear();
        return DC_OK;
    }
    if (H < 1 || W < 1 || !tuning_ok(t)) return DC_ERR_INVALID_ARG;
    return put_class(ctx, H, W, Tuning{t->a_warps_per_sm, t->b_ctas_per_sm, t->b_sparse_fill, t->a_strip_cols},
                     false);
}

dc_status dc_get_tuning(const dc_ctx* ctx, dc_tuning* t)
{
    if (!ctx || !t) return DC_ERR_INVALID_ARG;
    t->a_warps_per_sm = ctx->tune.a_warps_per_sm;
    t->b_ctas_per_sm = ctx->tune.b_ctas_per_sm;
    t->b_sparse_fill = ctx->tune.b_sparse_fill;
    t->a_strip_cols = ctx->tune.a_strip_cols;
    return DC_OK;
}

dc_status dc_autotune(dc_ctx* ctx, const float* in, float* out, int n, int H, int W, const dc_params* params,
                      void* stream, dc_tuning* best)
{
    if (!ctx || !best || n < 1) return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return DC_ERR_CUDA;
    }
    const Tuning saved = ctx->tune;
    dc_status s = DC_OK;
    ctx->classes_off = true;  // every candidate's threshold applies to every frame
    // time one tuning: a warm-up call (which also checks the arguments), then three
    auto measure = [&](Tuning t, float* ms) -> dc_status {
        ctx->tune = t;
        dc_status r = dc_complete_uniform(ctx, in, out, n, H, W, params, stream);
        if (r != DC_OK) return r;
        cudaEventRecord(e0, st);
        for (int k = 0; k < 3 && r == DC_OK; ++k) r = dc_complete_uniform(ctx, in, out, n, H, W, params, stream);
        cudaEventRecord(e1, st);
        if (r != DC_OK) return r;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            return DC_ERR_CUDA;
        return DC_OK;
    };
    // coordinate descent: each knob in turn over its candidates, the others fixed
    static const int a_cand[] = {2, 3, 4, 6, 8, 12, 16, 24};
    static const int b_cand[] = {1, 2, 3, 4, 5};
    static const int f_cand[] = {0, 4, 8, 16, 32, 64, 160};
    static const int c_cand[] = {128, 64};
    Tuning best_t = saved;
    float best_ms = 1e30f;
    s = measure(best_t, &best_ms);
    for (int round = 0; round < 2 && s == DC_OK; ++round) {
        for (int a : a_cand) {
            float ms;
            if ((s = measure(Tuning{a, best_t.b_ctas_per_sm, best_t.b_sparse_fill, best_t.a_strip_cols}, &ms)) !=
                DC_OK)
                break;
            if (ms < best_ms) { best_ms = ms; best_t.a_warps_per_sm = a; }
        }
        for (int b : b_cand) {
            float ms;
            if (s != DC_OK || (s = measure(Tuning{best_t.a_warps_per_sm, b, best_t.b_sparse_fill, best_t.a_strip_cols},
                                           &ms)) != DC_OK)
                break;
            if (ms < best_ms) { best_ms = ms; best_t.b_ctas_per_sm = b; }
        }
        for (int f : f_cand) {
            float ms;
            if (s != DC_OK || (s = measure(Tuning{best_t.a_warps_per_sm, best_t.b_ctas_per_sm, f, best_t.a_strip_cols},
                                           &ms)) != DC_OK)
                break;
            if (ms < best_ms) { best_ms = ms; best_t.b_sparse_fill = f; }
        }
        for (int c : c_cand) {
            float ms;
            if (s != DC_OK || (s = measure(Tuning{best_t.a_warps_per_sm, best_t.b_ctas_per_sm, best_t.b_sparse_fill, c},
                                           &ms)) != DC_OK)
                break;
            if (ms < best_ms) { best_ms = ms; best_t.a_strip_cols = c; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->classes_off = false;
    ctx->tune = (s == DC_OK) ? best_t : saved;
    if (s == DC_OK) s = put_class(ctx, H, W, best_t, true);
    best->a_warps_per_sm = ctx->tune.a_warps_per_sm;
    best->b_ctas_per_sm = ctx->tune.b_ctas_per_sm;
    best->b_sparse_fill = ctx->tune.b_sparse_fill;
    best->a_strip_cols = ctx->tune.a_strip_cols;
    return s;
}

dc_status dc_set_profiling(dc_ctx* ctx, int every)
{
    if (!ctx || every < 0) return DC_ERR_INVALID_ARG;
    const bool on = every > 0;
    DeviceGuard g(ctx->device);
    if (on && !ctx->prof_ev) {
        ctx->prof_ev = new (std::nothrow) cudaEvent_t[3 * DC_PROFILE_CALLS]();
        if (!ctx->prof_ev) return DC_ERR_OOM;
        for (int i = 0; i < 3 * DC_PROFILE_CALLS; ++i)
            if (cudaEventCreate(&ctx->prof_ev[i]) != cudaSuccess) { cudaGetLastError(); return DC_ERR_CUDA; }
    }
    ctx->profiling = on;
    ctx->prof_every = on ? every : 1;
    ctx->prof_tick = 0;
    ctx->prof_next = 0;
    ctx->prof_count = 0;
    return DC_OK;
}

dc_status dc_set_graph_cache(dc_ctx* ctx, int max_graphs)
{
    if (!ctx || max_graphs < 0 || max_graphs > DC_MAX_GRAPHS) return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (max_graphs != ctx->graph_max) {
        if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) return note(ctx, DC_ERR_CUDA);
        drop_graphs(ctx);
    }
    ctx->graph_max = max_graphs;
    return DC_OK;
}

int dc_graph_cache_entries(const dc_ctx* ctx) { return ctx ? (int)ctx->graphs.size() : 0; }

dc_status dc_kernel_times(dc_ctx* ctx, float* ms, int max_calls, int* n_out)
{
    if (!ctx || !ms || max_calls < 0 || !n_out) return DC_ERR_INVALID_ARG;
    *n_out = 0;
    if (!ctx->prof_ev || ctx->prof_count == 0) return DC_OK;
    DeviceGuard g(ctx->device);
    const int n = ctx->prof_count < max_calls ? ctx->prof_count : max_calls;
    int idx = (ctx->prof_next - n + DC_PROFILE_CALLS) % DC_PROFILE_CALLS;
    for (int i = 0; i < n; ++i, idx = (idx + 1) % DC_PROFILE_CALLS) {
        cudaEvent_t* ev = ctx->prof_ev + 3 * idx;
        float a = 0.0f, b = 0.0f;
        if (cudaEventSynchronize(ev[2]) != cudaSuccess || cudaEventElapsedTime(&a, ev[0], ev[1]) != cudaSuccess)
            return DC_ERR_CUDA;
        if (ctx->prof_has_b[idx] && cudaEventElapsedTime(&b, ev[1], ev[2]) != cudaSuccess) return DC_ERR_CUDA;
        ms[2 * i] = a;
        ms[2 * i + 1] = b;
    }
    *n_out = n;
    ctx->prof_next = 0;
    ctx->prof_count = 0;
    return DC_OK;
}

dc_status dc_last_async_error(dc_ctx* ctx)
{
    if (!ctx) return DC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    dc_status s = ctx->sticky;
    ctx->sticky = DC_OK;
    if (cudaStreamSynchronize(ctx->last_stream) != cudaSuccess) s = DC_ERR_CUDA;
    int waited_out = 0;
    if (ctx->err && cudaMemcpy(&waited_out, ctx->err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
        waited_out != 0) {
        cudaMemset(ctx->err, 0, sizeof(int));
        if (s == DC_OK) s = DC_ERR_TIMEOUT;
    }
    if (cudaGetLastError() != cudaSuccess) s = DC_ERR_CUDA;
    return s;
}

dc_status dc_inject_fault(dc_ctx* ctx, int fault)
{
    if (!ctx) return DC_ERR_INVALID_ARG;
    if (fault == DC_FAULT_WAIT) {
        DeviceGuard g(ctx->device);
        const int one = 1;
        if (cudaMemcpy(ctx->err, &one, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return DC_ERR_CUDA;
        return DC_OK;
    }
    if (fault == DC_FAULT_LAUNCH) {
        ctx->fail_next_launch = true;
        return DC_OK;
    }
    return DC_ERR_INVALID_ARG;
}

const char* dc_status_str(dc_status s)
{
    switch (s) {
    case DC_OK: return "DC_OK";
    case DC_ERR_INVALID_ARG: return "DC_ERR_INVALID_ARG";
    case DC_ERR_OOM: return "DC_ERR_OOM";
    case DC_ERR_CUDA: return "DC_ERR_CUDA";
    case DC_ERR_TIMEOUT: return "DC_ERR_TIMEOUT";
    case DC_ERR_UNSUPPORTED: return "DC_ERR_UNSUPPORTED";
    default: return "DC_ERR_UNKNOWN";
    }
}

void dc_destroy(dc_ctx* ctx)
{
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        cudaFree(ctx->c);
        cudaFree(ctx->ck);
        cudaFree(ctx->top);
        cudaFree(ctx->work);
        cudaFree(ctx->acc);
        cudaFree(ctx->table);
        cudaFree(ctx->err);
        drop_graphs(ctx);
        if (ctx->s_cap) cudaStreamDestroy(ctx->s_cap);
        if (ctx->done) cudaEventDestroy(ctx->done);
        for (int k = 0; k < 2; ++k) {
            cudaFree(ctx->io_in[k]);
            cudaFree(ctx->io_out[k]);
            if (ctx->io_read[k]) cudaEventDestroy(ctx->io_read[k]);
            if (ctx->io_drained[k]) cudaEventDestroy(ctx->io_drained[k]);
        }
        for (cudaEvent_t e : ctx->io_ev)
            if (e) cudaEventDestroy(e);
        if (ctx->s_in) cudaStreamDestroy(ctx->s_in);
        if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
        if (ctx->s_run) cudaStreamDestroy(ctx->s_run);
        if (ctx->prof_ev) {
            for (int i = 0; i < 3 * DC_PROFILE_CALLS; ++i)
                if (ctx->prof_ev[i]) cudaEventDestroy(ctx->prof_ev[i]);
            delete[] ctx->prof_ev;
        }
        cudaGetLastError();
    }
    delete ctx;
}

}  // extern "C"
