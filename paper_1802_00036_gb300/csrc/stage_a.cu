// stage_a.cu -- steps 1-4 of arXiv 1802.00036, Section IV, fused per tile.
//
// One CTA loads a kTileAH x kTileAW output tile plus a halo of
// R = r1 + 2 + 2 + 3 pixels (first element, close dilation, close erosion,
// 7x7 fill) into shared memory and runs the steps as passes over two
// ping-pong buffers.  Every pass computes the region its consumer reads;
// out-of-frame positions hold the neutral value of the consumer's operation
// (-inf before a max, +inf before a min), which is exactly "out-of-frame
// pixels are ignored".  The 5x5 and 7x7 squares are separable (row pass, then
// column pass); the first element is applied tap by tap from its shape.
//
// Output: C (step-4 map) into scratch, and for each column the smallest row
// whose C is non-empty via atomicMin on top[] (step 5 needs it).  With a
// stop before step 5 the tile is written straight to the output instead.
#include "common.cuh"

#include <climits>

namespace dcgb {
namespace {

template <int S> struct ShapeInfo;
template <> struct ShapeInfo<kDiamond5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kFull5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kCross5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kFull3> { static constexpr int r = 1; };
template <> struct ShapeInfo<kCircle5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kFull7> { static constexpr int r = 3; };

// Membership of offset (dy, dx) in the element (Fig. 4).
template <int S>
__device__ __forceinline__ constexpr bool in_shape(int dy, int dx)
{
    const int ay = dy < 0 ? -dy : dy, ax = dx < 0 ? -dx : dx;
    if (S == kDiamond5) return ay + ax <= 2;
    if (S == kFull5) return ay <= 2 && ax <= 2;
    if (S == kCross5) return (ay == 0 && ax <= 2) || (ax == 0 && ay <= 2);
    if (S == kFull3) return ay <= 1 && ax <= 1;
    if (S == kCircle5) return ay * ay + ax * ax <= 5;
    return ay <= 3 && ax <= 3;  // kFull7
}

template <int S>
__global__ void __launch_bounds__(kThreadsA)
stage_a_kernel(const FrameDesc* __restrict__ frames, int n_frames, int total_tiles, int stop,
               int* __restrict__ worklist)
{
    if (worklist && blockIdx.x == 0 && threadIdx.x == 0) worklist[0] = 0;
    constexpr int R1 = ShapeInfo<S>::r;
    constexpr int R = R1 + 2 + 2 + 3;
    constexpr int BH = kTileAH + 2 * R;
    constexpr int BW = kTileAW + 2 * R;
    constexpr int N = BH * BW;

    extern __shared__ float smem[];
    float* b0 = smem;
    float* b1 = smem + N;
    __shared__ int colmin[kTileAW];

    const int tid = threadIdx.x;

    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        __syncthreads();  // previous tile fully consumed
        const int f = find_frame<true>(frames, n_frames, t);
        const FrameDesc fd = frames[f];
        const int local = t - fd.base_a;
        const int ty = local / fd.tiles_x_a, tx = local - ty * fd.tiles_x_a;
        const int oy = ty * kTileAH - R, ox = tx * kTileAW - R;  // buffer origin
        const int H = fd.H, W = fd.W;
        auto inside = [&](int by, int bx) {
            const int y = oy + by, x = ox + bx;
            return y >= 0 && y < H && x >= 0 && x < W;
        };

        if (tid < kTileAW) colmin[tid] = INT_MAX;

        // P0, step 1: invert valid depths into b0; out-of-frame -> -inf
        for (int i = tid; i < N; i += kThreadsA) {
            const int by = i / BW, bx = i - by * BW;
            float v = ninf();
            if (inside(by, bx)) {
                const float d = fd.in[(size_t)(oy + by) * fd.in_pitch + (ox + bx)];
                v = (d >= kEmptyBelow) ? __fsub_rn(kInvertFrom, d) : 0.0f;
            }
            b0[i] = v;
        }
        __syncthreads();

        auto emit = [&](const float* buf) {  // write the tile region of buf to out
            for (int i = tid; i < kTileAH * kTileAW; i += kThreadsA) {
                const int ly = i / kTileAW, lx = i - ly * kTileAW;
                const int by = ly + R, bx = lx + R;
                if (inside(by, bx))
                    fd.out[(size_t)(oy + by) * fd.out_pitch + (ox + bx)] = buf[by * BW + bx];
            }
        };
        if (stop == kStopInvert) { emit(b0); continue; }

        // P1, step 2: first dilation b0 -> b1 on [R1, BH-R1) x [R1, BW-R1)
        for (int i = tid; i < N; i += kThreadsA) {
            const int by = i / BW, bx = i - by * BW;
            if (by < R1 || by >= BH - R1 || bx < R1 || bx >= BW - R1) continue;
            float m = ninf();
            if (inside(by, bx)) {
                m = b0[i];
#pragma unroll
                for (int dy = -R1; dy <= R1; ++dy)
#pragma unroll
                    for (int dx = -R1; dx <= R1; ++dx)
                        if (in_shape<S>(dy, dx)) m = fmaxf(m, b0[i + dy * BW + dx]);
            }
            b1[i] = m;
        }
        __syncthreads();
        if (stop == kStopDilate) { emit(b1); continue; }

        // P2, step 3a rows: max over 5 columns, b1 -> b0
        for (int i = tid; i < N; i += kThreadsA) {
            const int by = i / BW, bx = i - by * BW;
            if (by < R1 || by >= BH - R1 || bx < R1 + 2 || bx >= BW - R1 - 2) continue;
            float m = ninf();
            if (inside(by, bx)) {
                m = b1[i];
#pragma unroll
                for (int dx = -2; dx <= 2; ++dx) m = fmaxf(m, b1[i + dx]);
            }
            b0[i] = m;
        }
        __syncthreads();
        // P3, step 3a columns: max over 5 rows, b0 -> b1 (D; out-of-frame +inf)
        for (int i = tid; i < N; i += kThreadsA) {
            const int by = i / BW, bx = i - by * BW;
            if (by < R1 + 2 || by >= BH - R1 - 2 || bx < R1 + 2 || bx >= BW - R1 - 2) continue;
            float m = pinf();
            if (inside(by, bx)) {
                m = b0[i];
#pragma unroll
                for (int dy = -2; dy <= 2; ++dy) m = fmaxf(m, b0[i + dy * BW]);
            }
            b1[i] = m;
        }
        __syncthreads();
        // P4, step 3b rows: min over 5 columns, b1 -> b0
        for (int i = tid; i < N; i += kThreadsA) {
            const int by = i / BW, bx = i - by * BW;
            if (by < R1 + 2 || by >= BH - R1 - 2 || bx < R1 + 4 || bx >= BW - R1 - 4) continue;
            float m = pinf();
            if (inside(by, bx)) {
                m = b1[i];
#pragma unroll
                for (int dx = -2; dx <= 2; ++dx) m = fminf(m, b1[i + dx]);
            }
            b0[i] = m;
        }
        __syncthreads();
        // P5, step 3b columns: min over 5 rows, b0 -> b1 (B; out-of-frame -inf)
        for (int i = tid; i < N; i += kThreadsA) {
            const int by = i / BW, bx = i - by * BW;
            if (by < R1 + 4 || by >= BH - R1 - 4 || bx < R1 + 4 || bx >= BW - R1 - 4) continue;
            float m = ninf();
            if (inside(by, bx)) {
                m = b0[i];
#pragma unroll
                for (int dy = -2; dy <= 2; ++dy) m = fminf(m, b0[i + dy * BW]);
            }
            b1[i] = m;
        }
        __syncthreads();
        if (stop == kStopClose) { emit(b1); continue; }
        // P6, step 4 rows: max over 7 columns, b1 -> b0
        for (int i = tid; i < N; i += kThreadsA) {
            const int by = i / BW, bx = i - by * BW;
            if (by < R1 + 4 || by >= BH - R1 - 4 || bx < R || bx >= BW - R) continue;
            float m = ninf();
            if (inside(by, bx)) {
                m = b1[i];
#pragma unroll
                for (int dx = -3; dx <= 3; ++dx) m = fmaxf(m, b1[i + dx]);
            }
            b0[i] = m;
        }
        __syncthreads();
        // P7, step 4 columns + fill of empty pixels only: C on the tile
        const bool to_out = (stop == kStopFill7);
        for (int i = tid; i < kTileAH * kTileAW; i += kThreadsA) {
            const int ly = i / kTileAW, lx = i - ly * kTileAW;
            const int by = ly + R, bx = lx + R;
            if (!inside(by, bx)) continue;
            const int j = by * BW + bx;
            float c = b1[j];
            if (is_empty(c)) {
                float m = b0[j];
#pragma unroll
                for (int dy = -3; dy <= 3; ++dy) m = fmaxf(m, b0[j + dy * BW]);
                c = m;
            }
            const int y = oy + by, x = ox + bx;
            if (to_out) {
                fd.out[(size_t)y * fd.out_pitch + x] = c;
            } else {
                fd.c[(size_t)y * fd.c_pitch + x] = c;
                if (!is_empty(c)) atomicMin(&colmin[lx], y);
            }
        }
        if (!to_out) {
            __syncthreads();
            if (tid < kTileAW && colmin[tid] != INT_MAX) atomicMin(&fd.top[ox + R + tid], colmin[tid]);
        }
    }
}

template <int S>
cudaError_t launch_shape(const FrameDesc* d_frames, int n_frames, int total_tiles, int stop,
                         int* worklist, int sm_count, cudaStream_t stream)
{
    constexpr int R = ShapeInfo<S>::r + 7;
    const size_t smem = 2u * sizeof(float) * (kTileAH + 2 * R) * (kTileAW + 2 * R);
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(stage_a_kernel<S>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    int grid = total_tiles;
    const int cap = sm_count * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) return cudaSuccess;
    stage_a_kernel<S><<<grid, kThreadsA, smem, stream>>>(d_frames, n_frames, total_tiles, stop, worklist);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage_a(const FrameDesc* d_frames, int n_frames, int total_tiles, int shape,
                           int stop, int* worklist, int sm_count, cudaStream_t stream)
{
    switch (shape) {
    case kDiamond5: return launch_shape<kDiamond5>(d_frames, n_frames, total_tiles, stop, worklist, sm_count, stream);
    case kFull5: return launch_shape<kFull5>(d_frames, n_frames, total_tiles, stop, worklist, sm_count, stream);
    case kCross5: return launch_shape<kCross5>(d_frames, n_frames, total_tiles, stop, worklist, sm_count, stream);
    case kFull3: return launch_shape<kFull3>(d_frames, n_frames, total_tiles, stop, worklist, sm_count, stream);
    case kCircle5: return launch_shape<kCircle5>(d_frames, n_frames, total_tiles, stop, worklist, sm_count, stream);
    case kFull7: return launch_shape<kFull7>(d_frames, n_frames, total_tiles, stop, worklist, sm_count, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace dcgb
