// stage_b.cu -- steps 5-8 of arXiv 1802.00036, Section IV, fused per tile.
//
// One CTA loads a kTileBH x kTileBW output tile of the step-4 map C plus a
// halo of Rl + 4 pixels (step-6 half width, median 2, blur 2) into shared
// memory, applying step 5 on the fly: a pixel above its column's top row
// takes C(top, x), which is what copying the topmost value to the top of the
// frame produces.  Then, as passes over shared memory:
//   step 6  row max over 2 Rl + 1 columns, column max over 2 Rl + 1 rows,
//           written only into empty pixels (skipped when the tile's
//           median footprint holds no empty pixel -- the result is the same);
//   step 7  5x5 median with the border replicated, then the 5x5 binomial
//           Gaussian or the 13-tap bilateral with reflect-101 borders,
//           written only where the median output is non-empty;
//   step 8  100 - value where the median output is non-empty, 0 elsewhere.
#include "common.cuh"

namespace dcgb {
namespace {

// Median of 25 values: after pass i, v[i] is the (i+1)-th smallest, so
// v[12] is the median once passes 0..12 are done.  Compare-exchanges only.
__device__ __forceinline__ float median25(float (&v)[25])
{
#pragma unroll
    for (int i = 0; i <= 12; ++i)
#pragma unroll
        for (int j = i + 1; j < 25; ++j) {
            const float a = v[i], b = v[j];
            v[i] = fminf(a, b);
            v[j] = fmaxf(a, b);
        }
    return v[12];
}

// Mirror p into [0, n) without repeating the edge pixel (reflect-101).
__device__ __forceinline__ int reflect101(int p, int n)
{
    if (n == 1) return 0;
    while (p < 0 || p >= n) p = (p < 0) ? -p : 2 * (n - 1) - p;
    return p;
}

__device__ __forceinline__ int clampi(int p, int n) { return p < 0 ? 0 : (p >= n ? n - 1 : p); }

__global__ void __launch_bounds__(kThreadsB)
stage_b_kernel(const FrameDesc* __restrict__ frames, int n_frames, int total_tiles, StageBParams p)
{
    const int Rl = p.large_radius;
    const int R = Rl + 4;
    const int BH = kTileBH + 2 * R;
    const int BW = kTileBW + 2 * R;
    const int N = BH * BW;

    extern __shared__ float smem[];
    float* bE = smem;          // step 5 output E, then reused for nothing else
    float* bR = smem + N;      // step 6 row maxima, later the median output M
    float* bF = smem + 2 * N;  // step 6 output F
    int* ctop = reinterpret_cast<int*>(smem + 3 * N);      // BW entries
    float* cval = smem + 3 * N + BW;                        // BW entries

    const int tid = threadIdx.x;
    const float wn[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};  // [1 4 6 4 1]/16

    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        __syncthreads();
        const int f = find_frame<false>(frames, n_frames, t);
        const FrameDesc fd = frames[f];
        const int local = t - fd.base_b;
        const int ty = local / fd.tiles_x_b, tx = local - ty * fd.tiles_x_b;
        const int oy = ty * kTileBH - R, ox = tx * kTileBW - R;
        const int H = fd.H, W = fd.W;

        // column tops and their values for the buffer's columns
        for (int bx = tid; bx < BW; bx += kThreadsB) {
            const int x = ox + bx;
            int top = kNoTop;
            float v = 0.0f;
            if (p.extend_top && x >= 0 && x < W) {
                top = fd.top[x];
                if (top < H) v = fd.c[(size_t)top * fd.c_pitch + x];
                else top = kNoTop;
            }
            ctop[bx] = top;
            cval[bx] = v;
        }
        __syncthreads();

        // P0, step 5 applied while loading C: E; out-of-frame -> -inf
        for (int i = tid; i < N; i += kThreadsB) {
            const int by = i / BW, bx = i - by * BW;
            const int y = oy + by, x = ox + bx;
            float e = ninf();
            if (y >= 0 && y < H && x >= 0 && x < W) {
                const int top = ctop[bx];
                const bool above = (top != kNoTop) && y < top &&
                                   (p.extend_rows < 0 || y >= top - p.extend_rows);
                e = above ? cval[bx] : fd.c[(size_t)y * fd.c_pitch + x];
            }
            bE[i] = e;
        }
        __syncthreads();

        auto emit = [&](const float* buf) {
            for (int i = tid; i < kTileBH * kTileBW; i += kThreadsB) {
                const int ly = i / kTileBW, lx = i - ly * kTileBW;
                const int y = oy + R + ly, x = ox + R + lx;
                if (y < H && x < W) fd.out[(size_t)y * fd.out_pitch + x] = buf[(ly + R) * BW + lx + R];
            }
        };
        if (p.stop == kStopExtend) { emit(bE); continue; }

        // Is any pixel the median will read empty?  (T + 4, clipped)
        int any_empty = 0;
        if (p.large_fill_on) {
            for (int i = tid; i < N; i += kThreadsB) {
                const int by = i / BW, bx = i - by * BW;
                const int y = oy + by, x = ox + bx;
                if (by >= Rl && by < BH - Rl && bx >= Rl && bx < BW - Rl &&
                    y >= 0 && y < H && x >= 0 && x < W && is_empty(bE[i]))
                    any_empty = 1;
            }
        }
        any_empty = __syncthreads_or(any_empty);

        const float* bFill = bE;
        if (any_empty) {
            // P1, step 6 rows on rows [0, BH), cols [Rl, BW - Rl)
            for (int i = tid; i < N; i += kThreadsB) {
                const int by = i / BW, bx = i - by * BW;
                if (bx < Rl || bx >= BW - Rl) continue;
                const int y = oy + by, x = ox + bx;
                float m = ninf();
                if (y >= 0 && y < H && x >= 0 && x < W) {
                    for (int dx = -Rl; dx <= Rl; ++dx) m = fmaxf(m, bE[i + dx]);
                }
                bR[i] = m;
            }
            __syncthreads();
            // P2, step 6 columns, empty pixels only: F on [Rl, BH-Rl) x [Rl, BW-Rl)
            for (int i = tid; i < N; i += kThreadsB) {
                const int by = i / BW, bx = i - by * BW;
                if (by < Rl || by >= BH - Rl || bx < Rl || bx >= BW - Rl) continue;
                float e = bE[i];
                if (is_empty(e)) {
                    float m = e;
                    for (int dy = -Rl; dy <= Rl; ++dy) m = fmaxf(m, bR[i + dy * BW]);
                    e = m;
                }
                bF[i] = e;
            }
            __syncthreads();
            bFill = bF;
        }
        if (p.stop == kStopFillLarge) { emit(bFill); continue; }

        // P3, step 7 median on T + 2 (in frame), border replicated -> bR (M)
        const float* bMed = bFill;
        if (p.median) {
            const int lo = R - 2, hiy = BH - R + 2, hix = BW - R + 2;
            for (int i = tid; i < N; i += kThreadsB) {
                const int by = i / BW, bx = i - by * BW;
                if (by < lo || by >= hiy || bx < lo || bx >= hix) continue;
                const int y = oy + by, x = ox + bx;
                if (y < 0 || y >= H || x < 0 || x >= W) continue;
                float v[25];
#pragma unroll
                for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
                    for (int dx = -2; dx <= 2; ++dx) {
                        const int yy = clampi(y + dy, H) - oy, xx = clampi(x + dx, W) - ox;
                        v[(dy + 2) * 5 + dx + 2] = bFill[yy * BW + xx];
                    }
                bR[i] = median25(v);
            }
            __syncthreads();
            bMed = bR;
        }
        if (p.stop == kStopMedian) { emit(bMed); continue; }

        // P4, step 7 blur and step 8 inversion on the tile
        for (int i = tid; i < kTileBH * kTileBW; i += kThreadsB) {
            const int ly = i / kTileBW, lx = i - ly * kTileBW;
            const int y = oy + R + ly, x = ox + R + lx;
            if (y >= H || x >= W) continue;
            const float m = bMed[(ly + R) * BW + lx + R];
            float g = m;
            if (!is_empty(m)) {
                if (p.blur == kBlurGauss) {
                    float acc = 0.0f;
#pragma unroll
                    for (int dy = -2; dy <= 2; ++dy) {
                        const int yy = reflect101(y + dy, H) - oy;
                        float row = 0.0f;
#pragma unroll
                        for (int dx = -2; dx <= 2; ++dx) {
                            const int xx = reflect101(x + dx, W) - ox;
                            row = fmaf(wn[dx + 2], bMed[yy * BW + xx], row);
                        }
                        acc = fmaf(wn[dy + 2], row, acc);
                    }
                    g = acc;
                } else if (p.blur == kBlurBilateral) {
                    float num = 0.0f, den = 0.0f;
#pragma unroll
                    for (int dy = -2; dy <= 2; ++dy) {
                        const int yy = reflect101(y + dy, H) - oy;
#pragma unroll
                        for (int dx = -2; dx <= 2; ++dx) {
                            const int r2 = dy * dy + dx * dx;
                            if (r2 > 4) continue;
                            const int xx = reflect101(x + dx, W) - ox;
                            const float v = bMed[yy * BW + xx];
                            const float diff = v - m;
                            const float w = p.ws[r2] * expf(-(diff * diff) * p.inv_2sc2);
                            num = fmaf(v, w, num);
                            den += w;
                        }
                    }
                    g = num / den;
                }
            }
            float o;
            if (p.stop == kStopBlur) o = g;
            else o = is_empty(m) ? 0.0f : __fsub_rn(kInvertFrom, g);
            fd.out[(size_t)y * fd.out_pitch + x] = o;
        }
    }
}

}  // namespace

size_t stage_b_smem_bytes(int large_radius)
{
    const int R = large_radius + 4;
    const size_t BH = kTileBH + 2 * R, BW = kTileBW + 2 * R;
    return sizeof(float) * (3 * BH * BW + 2 * BW);
}

cudaError_t launch_stage_b(const FrameDesc* d_frames, int n_frames, int total_tiles,
                           const StageBParams& p, int sm_count, cudaStream_t stream)
{
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(stage_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)stage_b_smem_bytes(kMaxLargeFill / 2));
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    int grid = total_tiles;
    const int cap = sm_count * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) return cudaSuccess;
    stage_b_kernel<<<grid, kThreadsB, stage_b_smem_bytes(p.large_radius), stream>>>(
        d_frames, n_frames, total_tiles, p);
    return cudaGetLastError();
}

}  // namespace dcgb
