// stage_a.cu -- the float kernel of steps 1-4 (arXiv 1802.00036, Section
// IV): every unit of a stop before step 5, each a warp running the float
// unit of stage_a_float.cuh; and the strip and band geometry shared with
// the key kernel.
#include "stage_a_float.cuh"

namespace dcgb {
namespace {

using afloat::stage_a_unit;

// Persistent: warp w of the grid starts with unit w and then takes the next
// unclaimed unit from work[2] (zeroed before the launch), so SMs that drew
// cheap units (mostly empty rows) take more.  Unit 0 also zeroes work[0]
// and work[1] for stage B.
template <int S>
__global__ void __launch_bounds__(kThreadsA, kStageAFloatWarpsPerSM)
stage_a_stream(const FrameDesc* __restrict__ frames, int n_frames, int total_units, int stop,
               int* __restrict__ work, int band_stride)
{
    wait_previous_kernel();  // the frame table, the reset tops and counter
    allow_next_kernel();
    const int lane = threadIdx.x & 31;
    int unit = blockIdx.x * (kThreadsA / 32) + (threadIdx.x >> 5);
    if (unit == 0 && lane < 2) work[lane] = 0;  // step-6 count, stage-B tile counter
    const int warps = gridDim.x * (kThreadsA / 32);
    while (unit < total_units) {  // whole warps only
        stage_a_unit<S>(frames, n_frames, unit, stop, band_stride);
        int next = 0;
        if (lane == 0) next = atomicAdd(work + 2, 1);
        unit = warps + __shfl_sync(0xffffffffu, next, 0);
    }
}

template <int S>
cudaError_t launch_shape(const FrameDesc* d_frames, int n_frames, int total_units, int stop, int* work,
                         int band_stride, int sm_count, cudaStream_t stream)
{
    const int per_block = kThreadsA / 32;
    int grid = (total_units + per_block - 1) / per_block;
    // one-warp CTAs, as many per SM as the registers allow, persistent
    if (grid > kStageAFloatWarpsPerSM * sm_count) grid = kStageAFloatWarpsPerSM * sm_count;
    if (grid < 1) return cudaSuccess;
    return launch_after_previous(stage_a_stream<S>, dim3(grid), dim3(kThreadsA), 0, stream, d_frames, n_frames,
                                 total_units, stop, work, band_stride);
}

}  // namespace

cudaError_t preload_stage_a()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, stage_a_stream<kDiamond5>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_stream<kFull5>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_stream<kCross5>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_stream<kFull3>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_stream<kCircle5>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_stream<kFull7>);
    return e;
}

int stage_a_halo(int shape)
{
    return shape == kFull3 ? 8 : (shape == kFull7 ? 10 : 9);
}

int stage_a_strip_width(int shape, int strip_cols) { return strip_cols - 2 * stage_a_halo(shape); }

int stage_a_strips(int W, int shape, int strip_cols)
{
    const int ow = stage_a_strip_width(shape, strip_cols), h = stage_a_halo(shape);
    const int n = (W - h + ow - 1) / ow;
    return n < 1 ? 1 : n;
}

int stage_a_band_rows(int H, long long total_strips, long long target_warps)
{
    const long long target = target_warps > 0 ? target_warps : 1;
    long long bands = total_strips > 0 ? (target + total_strips - 1) / total_strips : 1;
    if (bands < 1) bands = 1;
    long long rows = (H + bands - 1) / bands;
    // short bands cost halo rows but shorten each warp's stream: a small batch
    // (one frame: ~120 units for ~1800 warp slots) finishes sooner
    if (rows < 6) rows = 6;
    return (int)rows;
}

cudaError_t launch_stage_a(const FrameDesc* d_frames, int n_frames, int total_units, int shape, int stop,
                           int* work, int band_stride, int sm_count, cudaStream_t stream)
{
    switch (shape) {
    case kDiamond5: return launch_shape<kDiamond5>(d_frames, n_frames, total_units, stop, work, band_stride, sm_count, stream);
    case kFull5: return launch_shape<kFull5>(d_frames, n_frames, total_units, stop, work, band_stride, sm_count, stream);
    case kCross5: return launch_shape<kCross5>(d_frames, n_frames, total_units, stop, work, band_stride, sm_count, stream);
    case kFull3: return launch_shape<kFull3>(d_frames, n_frames, total_units, stop, work, band_stride, sm_count, stream);
    case kCircle5: return launch_shape<kCircle5>(d_frames, n_frames, total_units, stop, work, band_stride, sm_count, stream);
    case kFull7: return launch_shape<kFull7>(d_frames, n_frames, total_units, stop, work, band_stride, sm_count, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dcgb
