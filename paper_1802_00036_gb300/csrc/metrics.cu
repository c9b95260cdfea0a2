// metrics.cu -- accuracy of completed depth maps against ground truth, the
// KITTI depth-completion measures the paper reports (Section V, Tables 1-3):
// RMSE and MAE in mm, iRMSE and iMAE in 1/km, over pixels whose ground
// truth is valid (>= 0.1 m); an empty prediction (< 0.1) has inverse 0.
//
// One pass over both maps: per thread float partial sums over a few pixels,
// then double sums across the warp, the block and (atomically) the frame.
#include "common.cuh"

namespace dcgb {
namespace {

constexpr int kMetricThreads = 256;
constexpr int kPixelsPerThread = 32;

__global__ void __launch_bounds__(kMetricThreads)
metrics_sum(const float* __restrict__ pred, const float* __restrict__ gt, long long frame_px, double* acc)
{
    const int f = blockIdx.y;
    const float* p = pred + (size_t)f * frame_px;
    const float* g = gt + (size_t)f * frame_px;
    float se = 0.0f, ae = 0.0f, ise = 0.0f, iae = 0.0f;
    int cnt = 0;
    const long long base = (long long)blockIdx.x * kMetricThreads * kPixelsPerThread + threadIdx.x;
#pragma unroll 4
    for (int k = 0; k < kPixelsPerThread; ++k) {
        const long long i = base + (long long)k * kMetricThreads;
        if (i >= frame_px) break;
        const float gv = __ldcs(g + i);
        if (!(gv >= kEmptyBelow)) continue;
        const float pv = __ldcs(p + i);
        const float ip = (pv >= kEmptyBelow) ? 1.0f / pv : 0.0f;
        const float d = pv - gv, id = ip - 1.0f / gv;
        se = fmaf(d, d, se);
        ae += fabsf(d);
        ise = fmaf(id, id, ise);
        iae += fabsf(id);
        ++cnt;
    }
    double v[5] = {se, ae, ise, iae, (double)cnt};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    __shared__ double part[kMetricThreads / 32][5];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int j = 0; j < 5; ++j) part[warp][j] = v[j];
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < kMetricThreads / 32; ++w) s += part[w][threadIdx.x];
        atomicAdd(acc + 5 * f + threadIdx.x, s);
    }
}

__global__ void metrics_finish(const double* __restrict__ acc, double* __restrict__ out, int n)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const double c = acc[5 * f + 4];
    double* o = out + 5 * f;
    if (c > 0.0) {
        o[0] = 1000.0 * sqrt(acc[5 * f + 0] / c);
        o[1] = 1000.0 * (acc[5 * f + 1] / c);
        o[2] = 1000.0 * sqrt(acc[5 * f + 2] / c);
        o[3] = 1000.0 * (acc[5 * f + 3] / c);
    } else {
        o[0] = o[1] = o[2] = o[3] = 0.0;
    }
    o[4] = c;
}

}  // namespace

cudaError_t preload_metrics()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, metrics_sum);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, metrics_finish);
    return e;
}

cudaError_t launch_metrics(const float* pred, const float* gt, int n, int H, int W, double* acc, double* out,
                           cudaStream_t stream)
{
    const long long px = (long long)H * W;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 5 * (size_t)n, stream);
    if (e != cudaSuccess) return e;
    const long long per_block = (long long)kMetricThreads * kPixelsPerThread;
    const dim3 grid((unsigned)((px + per_block - 1) / per_block), (unsigned)n);
    metrics_sum<<<grid, kMetricThreads, 0, stream>>>(pred, gt, px, acc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    metrics_finish<<<(n + 127) / 128, 128, 0, stream>>>(acc, out, n);
    return cudaGetLastError();
}

}  // namespace dcgb
