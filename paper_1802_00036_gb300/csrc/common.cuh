// common.cuh -- definitions shared by the libdc kernels and host code.
//
// Depth completion of arXiv 1802.00036, Section IV.  Two kernels split the
// chain where a whole-column dependency appears (step 5 needs the topmost
// non-empty row of every column after step 4):
//   stage A: steps 1-4 on halo'd tiles, writes the step-4 map C to scratch
//            and the per-column top row with atomicMin;
//   stage B: steps 5-8 on halo'd tiles of C, writes the output.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dc.h"

namespace dcgb {

// The checks every entry point applies to a dc_params (dc_api.cu).
bool params_ok(const dc_params* p);

// A pixel is empty below 0.1 (Section IV-1: empty pixels hold 0, valid
// inverted depths lie 20 m or more above them).
constexpr float kEmptyBelow = 0.1f;
// D_inv = 100 - D (Section IV-1 and IV-8).
constexpr float kInvertFrom = 100.0f;

// A column's top row as stage B keeps it (any real row is smaller).
constexpr int kNoTop = 0x7F7F7F7F;

// The step-4 map C between the kernels is kept as 16-bit keys: a value v
// that is k / 256 for an integer k (KITTI stores depth as 16-bit fixed
// point, depth x 256, and every such inverted depth stays on that grid
// through steps 1-4, which only select values) is stored as k, an exact,
// order-preserving encoding; any other value is stored as kKeyOff, with the
// value itself at the same position of a float map.  Inverted depths of
// valid inputs lie below 100, so a real key is at most kKeyMax.
constexpr unsigned kKeyOff = 0xFFFFu;
constexpr unsigned kKeyMax = 25600u;
// A key k is empty (k / 256 < 0.1) exactly when k <= 25.
constexpr unsigned kEmptyKeyMax = 25;

// 16-bit key of v: k with v == k / 256 exactly, k < 65536; `ok` is cleared
// when v has no such key.  fma(v, 256, 2^23) holds 2^23 + k exactly iff
// v * 256 is an integer in [0, 2^23): the nearest k is in its low mantissa
// bits, and rebuilding k / 256 from them gives v back only when v is on the
// grid and in [0, 256).
__device__ __forceinline__ unsigned key_of(float v, bool& ok)
{
    const unsigned k = __float_as_uint(fmaf(v, 256.0f, 8388608.0f)) & 0xFFFFu;
    ok = ok && (__uint_as_float(0x47000000u | k) - 32768.0f) == v;
    return k;
}

// The float value of a 16-bit key: exactly k / 256.
__device__ __forceinline__ float key_value(unsigned k)
{
    return __uint_as_float(0x47000000u | k) - 32768.0f;  // (2^15 + k / 256) - 2^15
}

// A column's top in scratch: the row in the high half, the key of the C
// value there (kKeyOff: the value is in the float map) in the low half, so
// that one 64-bit atomicMin keeps the smallest row with its value and one
// load brings both.
constexpr unsigned long long kNoTopPacked = ~0ull;
__device__ __forceinline__ unsigned long long top_pack(int row, unsigned key)
{
    return ((unsigned long long)(unsigned)row << 32) | (unsigned long long)key;
}

// Stage A: one warp streams one (strip, band) unit; one warp per block.
constexpr int kStageAColsPerLane = 4;
constexpr int kThreadsA = 32;  // one warp per CTA: the block scheduler spreads warps evenly
constexpr int kStageAFloatWarpsPerSM = 12;  // the float kernel's registers allow twelve per SM
constexpr int kStageAKeysWarpsPerSM = 16;   // the key kernel's
// Stage B output tile (median blocks of 2 x 8 over the tile + 2 ring).
constexpr int kTileBH = 60;
constexpr int kTileBW = 60;
constexpr int kThreadsB = 128;
// Stage B's region of C (tile + 4 ring) comes as one box of keys whose first
// column is rounded down to a multiple of 8 (16 bytes), hence 4 more columns.
constexpr int kKeyBoxW = kTileBW + 12;
constexpr int kKeyBoxH = kTileBH + 8;
static_assert(kTileBW % 8 == 4 || kTileBW % 8 == 0, "the region starts 0 or 4 columns into its key box");

// Largest step-6 square side the kernels accept.
constexpr int kMaxLargeFill = 63;

// Codes shared with include/dc.h.
enum Shape { kDiamond5 = 0, kFull5 = 1, kCross5 = 2, kFull3 = 3, kCircle5 = 4, kFull7 = 5 };
enum Blur { kBlurNone = 0, kBlurGauss = 1, kBlurBilateral = 2 };
enum Stop {
    kStopFull = 0, kStopInvert = 1, kStopDilate = 2, kStopClose = 3, kStopFill7 = 4,
    kStopExtend = 5, kStopFillLarge = 6, kStopMedian = 7, kStopBlur = 8
};

// One frame of a batch as the kernels see it.
struct FrameDesc {
    const float* in;   // sparse depth, in_pitch floats per row
    float* out;        // result, out_pitch floats per row
    unsigned short* ck;  // step-4 map as keys, c_pitch per row (scratch)
    float* c;          // step-4 values whose key is kKeyOff, c_pitch floats per row (scratch)
    unsigned long long* top;  // W entries: top_pack(topmost non-empty row of C, its key); kNoTopPacked: none
    int H, W;
    int in_pitch, out_pitch, c_pitch;  // c_pitch: a multiple of 32 elements
    int tiles_x_a, base_a;  // stage A: strips per frame, first flat unit
    int band_a;             // stage A: rows per band
    int ow_a;               // stage A: output columns per strip
    int tiles_x_b, base_b;  // stage B: same
    int sparse_fill;        // stage B: most empty pixels a tile of this frame fills itself (0..160)
};

// Runtime parameters of stage B.
struct StageBParams {
    int large_radius;   // step-6 half width; 0 with large_fill_on == 0
    int large_fill_on;
    int median;
    int blur;
    int extend_top;
    int extend_rows;    // < 0: unlimited
    int stop;
    int row_stride;       // frames of one shape: the batch's tiles per tile row (tile order), else 0
    int tma;              // 1: regions come by one tensor copy through the CUtensorMap of C (frames of one shape)
    int fill_inline;      // 1: the main pass runs step-6 worklist tiles itself (set by launch_stage_b)
    float ws[5];        // bilateral spatial weight for dy^2+dx^2 = 0,1,2,(3),4
    float inv_2sc2;     // 1 / (2 sigma_color^2)
};

__device__ __forceinline__ bool is_empty(float v) { return !(v >= kEmptyBelow); }

__device__ __forceinline__ float ninf() { return __int_as_float(0xff800000); }
__device__ __forceinline__ float pinf() { return __int_as_float(0x7f800000); }

// Programmatic dependent launch.  The stage kernels are launched so that the
// GPU may start them while the previous kernel of the stream is finishing;
// each first waits until that kernel has completed and its writes are
// visible (without the launch attribute the wait returns at once).  The
// kernel before lets them launch once all of its blocks have started: its
// grids are persistent (every block resident from the start), so the next
// kernel's blocks only take the room its finished blocks leave.
__device__ __forceinline__ void wait_previous_kernel() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_kernel() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_after_previous(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                         cudaStream_t stream, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// C at frame pixel (y, x) as a float.
__device__ __forceinline__ float c_at(const FrameDesc& fd, int y, int x)
{
    const size_t i = (size_t)y * fd.c_pitch + x;
    const unsigned k = fd.ck[i];
    return k == kKeyOff ? fd.c[i] : key_value(k);
}

// The value of a column top (row, key) of frame column x as a float.
__device__ __forceinline__ float top_value(const FrameDesc& fd, int row, unsigned key, int x)
{
    return key == kKeyOff ? fd.c[(size_t)row * fd.c_pitch + x] : key_value(key);
}

// Frame owning flat tile t: the last f with base(f) <= t.
template <bool kStageA>
__device__ __forceinline__ int find_frame(const FrameDesc* __restrict__ d, int n, int t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int b = kStageA ? d[mid].base_a : d[mid].base_b;
        if (b <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Stage A geometry (stage_a.cu): output columns per strip of strip_cols
// columns (128: four per lane; 64: two, the key kernel only) and the halo
// (= vertical delay) for a first element.
int stage_a_strip_width(int shape, int strip_cols);
int stage_a_strips(int W, int shape, int strip_cols);  // strips covering W columns (the first writes its left halo)
int stage_a_halo(int shape);
// Rows per stage-A band so that a batch with `total_strips` strips gives
// about `target_warps` warps; at least 6 rows.
int stage_a_band_rows(int H, long long total_strips, long long target_warps);

// Launch-shape choices (the results never depend on them).
struct Tuning {
    int a_warps_per_sm;   // stage A: warps in flight per SM the bands aim for
    int b_ctas_per_sm;    // stage B: persistent CTAs per SM (1..5)
    int b_sparse_fill;    // stage B: most empty pixels a tile fills itself (0..160)
    int a_strip_cols;     // stage A (on keys): strip width, 128 or 64 columns
};
constexpr Tuning kDefaultTuning{8, 5, 160, 128};

// Launchers (stage_a.cu, stage_b.cu).  Return cudaGetLastError().
// `work` holds 3 + (stage B tiles) ints: the number of stage-B tiles that
// need the step-6 kernel and the counter from which persistent stage-B CTAs
// take tiles (both zeroed by stage A), the counter from which stage-A warps
// take units (zeroed before stage A starts), then those tiles.  band_stride:
// the batch's strip count when all frames have one shape (units then go
// band by band over the whole batch, bottom bands first), else 0.
cudaError_t launch_stage_a(const FrameDesc* d_frames, int n_frames, int total_units,
                           int shape, int stop, int* work, int band_stride, int sm_count,
                           cudaStream_t stream);
// Steps 1-4 of the full chain on packed 16-bit keys (stage_a_keys.cu); the
// warp that meets a unit whose inputs are off the key grid redoes it on
// floats (stage_a_float.cuh).
cudaError_t launch_stage_a_keys(const FrameDesc* d_frames, int n_frames, int total_units, int shape, int strip_cols,
                                int* work, int band_stride, int sm_count, cudaStream_t stream);
// cmap: with p.tma, the tensor map of the batch's step-4 maps C as a
// W x H x n_frames array (rows c_pitch floats apart, frames H c_pitch);
// err: set to 1 when a bounded device-side wait gives up.
// ffill: the step-6 tiles off the key grid, ffill[0] of them from ffill[1]
// (ffill[0] zeroed before the call, room for every tile).
// Kernels one launch_stage_b call starts for these parameters.
int stage_b_launches(const StageBParams& p);
cudaError_t launch_stage_b(const FrameDesc* d_frames, int n_frames, int total_tiles,
                           const StageBParams& p, int* worklist, int* ffill, int sm_count, int ctas_per_sm,
                           const CUtensorMap* cmap, int* err, cudaStream_t stream);

// Load every kernel of a translation unit on the current device
// (cudaFuncGetAttributes on each), so that no later launch pays CUDA's lazy
// module loading; dc_create calls them all.
cudaError_t preload_stage_a();
cudaError_t preload_stage_a_keys();
cudaError_t preload_stage_b();
cudaError_t preload_metrics();
cudaError_t preload_project();

// Accuracy measures (metrics.cu): acc holds 5 n doubles of scratch, out
// (device) receives 5 n doubles.
cudaError_t launch_metrics(const float* pred, const float* gt, int n, int H, int W, double* acc, double* out,
                           cudaStream_t stream);

// LIDAR points to a sparse map (project.cu); P is a host array of 12 doubles.
cudaError_t launch_project(const float* xyz, long long n, const double* P, int H, int W, double d_min,
                           double d_max, float* depth, int pitch, cudaStream_t stream);

}  // namespace dcgb
