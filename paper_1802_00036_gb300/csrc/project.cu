// project.cu -- LIDAR points to a sparse depth map, the step before the
// chain (Section V: the benchmark projects the scans into the image with the
// camera calibration).  One thread per point: (u, v, w) = P (x, y, z, 1) in
// double with explicit round-to-nearest products and sums (no contraction,
// the order of the plain statement); a point with w > 0 in [d_min, d_max]
// lands in pixel (floor(v / w), floor(u / w)).  Each pixel keeps its nearest
// depth: positive floats order like their bit patterns, so an unsigned
// atomicMin on the bits does it; untouched pixels become 0.
#include "common.cuh"

namespace dcgb {
namespace {

struct Proj {
    double p[12];
};

constexpr unsigned kFar = 0x7F7F7F7Fu;  // memset pattern, above any depth's bits

__global__ void project_points(const float* __restrict__ xyz, long long n, Proj P, int H, int W, double d_min,
                               double d_max, unsigned* __restrict__ bits, int pitch)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    auto row = [&](int r) {
        double s = __dmul_rn(P.p[4 * r + 0], x);
        s = __dadd_rn(s, __dmul_rn(P.p[4 * r + 1], y));
        s = __dadd_rn(s, __dmul_rn(P.p[4 * r + 2], z));
        return __dadd_rn(s, P.p[4 * r + 3]);
    };
    const double u = row(0), v = row(1), w = row(2);
    if (!(w > 0.0) || w < d_min || w > d_max) return;
    const double col = floor(__ddiv_rn(u, w)), rr = floor(__ddiv_rn(v, w));
    if (!(col >= 0.0 && col < W && rr >= 0.0 && rr < H)) return;
    const float d = __double2float_rn(w);
    atomicMin(bits + (size_t)rr * pitch + (long long)col, __float_as_uint(d));
}

__global__ void far_to_empty(unsigned* __restrict__ bits, int H, int W, int pitch)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)H * W) return;
    const long long r = i / W, c = i - r * W;
    unsigned* b = bits + r * pitch + c;
    if (*b == kFar) *b = 0u;  // the bits of 0.0f
}

}  // namespace

cudaError_t preload_project()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, project_points);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, far_to_empty);
    return e;
}

cudaError_t launch_project(const float* xyz, long long n, const double* P, int H, int W, double d_min,
                           double d_max, float* depth, int pitch, cudaStream_t stream)
{
    cudaError_t e = cudaMemset2DAsync(depth, (size_t)pitch * sizeof(float), 0x7F, (size_t)W * sizeof(float), H,
                                      stream);
    if (e != cudaSuccess) return e;
    Proj pm;
    for (int k = 0; k < 12; ++k) pm.p[k] = P[k];
    unsigned* bits = reinterpret_cast<unsigned*>(depth);
    if (n > 0) {
        project_points<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(xyz, n, pm, H, W, d_min, d_max, bits, pitch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const long long px = (long long)H * W;
    far_to_empty<<<(unsigned)((px + 255) / 256), 256, 0, stream>>>(bits, H, W, pitch);
    return cudaGetLastError();
}

}  // namespace dcgb
