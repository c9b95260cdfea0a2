// noalloc.cu -- dc_complete_noalloc: the chain without any run-time device
// allocation.  The paper has no counterpart; see include/dc.h for who needs it.
//
// All scratch (frame table, per-column tops, step-4 map) sits in one
// file-scope device array.  Host code must not use the array's name as a
// pointer: here it is only a host-side stand-in, and a kernel handed it would
// fault or read the wrong memory.  The device address is looked up on each
// call with cudaGetSymbolAddress, with the caller's device current.
#include "../../include/dc.h"
#include "common.cuh"

#include <cmath>
#include <cstdint>
#include <mutex>

using namespace dcgb;

namespace {

constexpr size_t kTableBytes = 65536;
constexpr size_t kTopBytes = 8u * DC_NOALLOC_MAX_COLUMNS;
constexpr size_t kWorkBytes = 4u * DC_NOALLOC_WORK_INTS;
constexpr size_t kKeyBytes = 2u * DC_NOALLOC_MAX_PIXELS;
constexpr size_t kMapBytes = 4u * DC_NOALLOC_MAX_PIXELS;
static_assert(kTableBytes + kTopBytes + kWorkBytes + kKeyBytes + kMapBytes == DC_NOALLOC_SCRATCH_BYTES, "layout");
static_assert(DC_NOALLOC_MAX_FRAMES * sizeof(FrameDesc) <= kTableBytes, "frame table");

// Layout: [frame table | tops | worklist | step-4 keys | step-4 values];
// each part 256-byte aligned.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int g_sm_count[kMaxDevices] = {};  // per device, looked up once

// The array's device address in the current context (looked up on every
// call: a cached address would go stale under another context of the same
// device or after a device reset) and the device's SM count; must run with
// `dev` current.
dc_status setup(int dev, unsigned char** ptr, int* sms)
{
    if (dev < 0 || dev >= kMaxDevices) return DC_ERR_UNSUPPORTED;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_sm_count[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return DC_ERR_CUDA;
        }
        g_sm_count[dev] = n;
    }
    *ptr = static_cast<unsigned char*>(p);
    *sms = g_sm_count[dev];
    return DC_OK;
}

// Writes the frame table for n packed frames, resets the tops and stage A's
// unit counter: the only preparation the two stage kernels need, done on
// the device so that the call copies nothing from the host.
__global__ void noalloc_prepare(FrameDesc* table, unsigned long long* top, unsigned short* ckeys, float* cmap,
                                const float* in, float* out,
                                int n, int H, int W, int c_pitch, int tiles_x_a, int ow_a, int tiles_a, int band_a,
                                int tiles_x_b, int tiles_b, int top_ints, int* counter, int* ffill, int* err)
{
    allow_next_kernel();  // stage A may launch; it waits for this kernel's writes
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (tid == 0) *ffill = 0;        // stage B's float step-6 list: length
    if (tid == 0) {
        *counter = 0;  // stage A's unit counter
        *err = 0;      // stage B's error word (set only by its tensor-copy wait, which this path does not use)
    }
    for (int i = tid; i < n; i += stride) {
        FrameDesc d;
        d.in = in + (size_t)i * H * W;
        d.out = out + (size_t)i * H * W;
        d.c = cmap ? cmap + (size_t)i * H * c_pitch : nullptr;
        d.ck = ckeys ? ckeys + (size_t)i * H * c_pitch : nullptr;
        d.top = top ? top + (size_t)i * c_pitch : nullptr;
        d.H = H;
        d.W = W;
        d.in_pitch = W;
        d.out_pitch = W;
        d.c_pitch = c_pitch;
        d.tiles_x_a = tiles_x_a;
        d.base_a = i * tiles_a;
        d.band_a = band_a;
        d.ow_a = ow_a;
        d.tiles_x_b = tiles_x_b;
        d.base_b = i * tiles_b;
        d.sparse_fill = kDefaultTuning.b_sparse_fill;
        table[i] = d;
    }
    if (top)
        for (int i = tid; i < top_ints; i += stride) top[i] = kNoTopPacked;
}


}  // namespace

extern "C" dc_status dc_complete_noalloc(const float* in, float* out, int n, int H, int W,
                                         const dc_params* params, void* stream)
{
    if (n < 0 || !params_ok(params)) return DC_ERR_INVALID_ARG;
    if (n == 0) return DC_OK;
    if (!in || !out || H < 1 || W < 1) return DC_ERR_INVALID_ARG;
    if (((uintptr_t)in % sizeof(float)) != 0 || ((uintptr_t)out % sizeof(float)) != 0)
        return DC_ERR_INVALID_ARG;
    const size_t span = (size_t)n * H * W * sizeof(float);
    if ((uintptr_t)in < (uintptr_t)out + span && (uintptr_t)out < (uintptr_t)in + span)
        return DC_ERR_INVALID_ARG;
    const size_t c_pitch = ((size_t)W + 31) / 32 * 32;
    if (n > DC_NOALLOC_MAX_FRAMES || (size_t)n * H * c_pitch > (size_t)DC_NOALLOC_MAX_PIXELS ||
        (size_t)n * c_pitch > (size_t)DC_NOALLOC_MAX_COLUMNS)
        return DC_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return DC_ERR_CUDA; }
    unsigned char* base = nullptr;
    int sms = 0;
    dc_status s = setup(dev, &base, &sms);
    if (s != DC_OK) return s;

    FrameDesc* table = reinterpret_cast<FrameDesc*>(base);
    unsigned long long* top = reinterpret_cast<unsigned long long*>(base + kTableBytes);
    int* work = reinterpret_cast<int*>(base + kTableBytes + kTopBytes);
    unsigned short* ckeys = reinterpret_cast<unsigned short*>(base + kTableBytes + kTopBytes + kWorkBytes);
    float* cmap = reinterpret_cast<float*>(base + kTableBytes + kTopBytes + kWorkBytes + kKeyBytes);
    const bool need_b = (params->stop_after == DC_STOP_FULL || params->stop_after >= DC_STOP_EXTEND);
    const int strip_cols = kDefaultTuning.a_strip_cols;
    const int tiles_x_a = stage_a_strips(W, params->first_kernel, strip_cols);
    const int ow_a = stage_a_strip_width(params->first_kernel, strip_cols);
    const int band_a = stage_a_band_rows(H, (long long)tiles_x_a * n,
                                         (long long)kDefaultTuning.a_warps_per_sm * sms);
    const int tiles_a = tiles_x_a * ((H + band_a - 1) / band_a);
    const int tiles_x_b = (W + kTileBW - 1) / kTileBW;
    const int tiles_b = tiles_x_b * ((H + kTileBH - 1) / kTileBH);
    // work: three counters, the step-6 tile list, the float step-6 list (a
    // count and the tiles), the error word last
    if ((long long)tiles_a * n > INT32_MAX / 2 || 2 * (long long)tiles_b * n + 4 + 1 > DC_NOALLOC_WORK_INTS)
        return DC_ERR_UNSUPPORTED;
    int* ffill = work + 3 + (size_t)tiles_b * n;
    cudaStream_t st = (cudaStream_t)stream;

    const int top_ints = need_b ? (int)((size_t)n * c_pitch) : 0;
    const int threads = 256;
    int blocks = (top_ints > n ? top_ints : n) / threads + 1;
    if (blocks > 1024) blocks = 1024;
    noalloc_prepare<<<blocks, threads, 0, st>>>(table, need_b ? top : nullptr, need_b ? ckeys : nullptr,
                                                 need_b ? cmap : nullptr,
                                                 in, out, n, H, W, (int)c_pitch, tiles_x_a, ow_a, tiles_a, band_a,
                                                 tiles_x_b, tiles_b, top_ints, work + 2, ffill,
                                                 work + DC_NOALLOC_WORK_INTS - 1);
    if (cudaGetLastError() != cudaSuccess) return DC_ERR_CUDA;

    const int stop_a = need_b ? kStopFull : params->stop_after;
    if (need_b) {  // steps 1-4 on keys (a unit off the key grid on floats, by the same warp)
        if (launch_stage_a_keys(table, n, tiles_a * n, params->first_kernel, strip_cols, work, tiles_x_a * n, sms,
                                st) != cudaSuccess)
            return DC_ERR_CUDA;
    } else if (launch_stage_a(table, n, tiles_a * n, params->first_kernel, stop_a, work, tiles_x_a * n, sms, st) !=
               cudaSuccess) {
        return DC_ERR_CUDA;
    }
    if (need_b) {
        StageBParams bp{};
        bp.large_fill_on = params->large_fill_on ? 1 : 0;
        bp.large_radius = params->large_fill_on ? params->large_fill / 2 : 0;
        bp.median = params->median ? 1 : 0;
        bp.blur = params->blur;
        bp.extend_top = params->extend_top ? 1 : 0;
        bp.extend_rows = params->extend_rows;
        bp.stop = params->stop_after;
        bp.row_stride = tiles_x_b * n;
        const double ss = params->blur == DC_BLUR_BILATERAL ? params->sigma_space : 1.0;
        const double sc = params->blur == DC_BLUR_BILATERAL ? params->sigma_color : 1.0;
        for (int r2 = 0; r2 < 5; ++r2) bp.ws[r2] = (float)std::exp(-(double)r2 / (2.0 * ss * ss));
        bp.inv_2sc2 = (float)(1.0 / (2.0 * sc * sc));
        // regions by cp.async (no tensor map: the map would have to be written
        // for the array's address); the error word is zeroed by noalloc_prepare
        if (launch_stage_b(table, n, tiles_b * n, bp, work, ffill, sms, kDefaultTuning.b_ctas_per_sm, nullptr,
                           work + DC_NOALLOC_WORK_INTS - 1, st) != cudaSuccess)
            return DC_ERR_CUDA;
    }
    return DC_OK;
}
