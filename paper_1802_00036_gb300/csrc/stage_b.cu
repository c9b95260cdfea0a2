// stage_b.cu -- steps 5-8 of arXiv 1802.00036, Section IV, fused per tile.
//
// Output tile kTBH x kTBW.  Phase 1 (persistent CTAs) brings the step-4 map
// C over the tile plus a 4-pixel ring (median 2 + blur 2) into shared memory
// with cp.async and applies step 5 in place (a pixel above
// its column's top row takes C(top, x), which is what copying the topmost
// value to row 0 gives).  Step 6 changes only empty pixels: a tile with a
// few of them in that region fills each with one warp (the maximum over its
// (2 Rl + 1)^2 window, read from C); a tile with many goes on a worklist for
// phase 2, which loads the wider ring, takes row then column maxima and
// fills the empty pixels.  The frame border is replicated around the region
// (the median's rule).  Then:
//   step 7  5x5 median on the tile + 2 ring by the generated network of
//           median_net.cuh, two 2 x 8 output blocks per thread.  When every
//           value of the tile is k/256 m for an integer k < 65536 (KITTI
//           stores depth as 16-bit fixed point, depth x 256), the values are
//           replaced by their 16-bit keys k -- an exact, order-preserving
//           encoding -- and both blocks run at once in the two halves of
//           32-bit registers (packed min/max, 3-input); otherwise the float
//           network runs per block.  The ring is mirrored (reflect-101) for
//           the blur; then the Gaussian [1 4 6 4 1]/16 as a row pass and a
//           column pass (FMA chains, dyadic weights), or the 13-tap
//           bilateral; both only where the median is non-empty;
//   step 8  100 - value where the median is non-empty, 0 elsewhere.
#include "common.cuh"
#include "median_net.cuh"

namespace dcgb {
namespace {

constexpr int kTBH = kTileBH;       // output tile rows
constexpr int kTBW = kTileBW;       // output tile columns
constexpr int kMR = kTBH + 4;       // median region rows (tile + 2 ring)
constexpr int kMC = kTBW + 4;       // median region columns
constexpr int kER = kTBH + 8;       // median input rows (tile + 4 ring)
constexpr int kEC = kTBW + 8;       // median input columns
constexpr int kES = kEC;            // stride of the median input buffers
constexpr int kMS = kMC;            // stride of the median output buffer
constexpr int kRS = kTBW;           // stride of the Gaussian row-pass buffer
constexpr int kHalf = kMR / 2;      // median-region rows per block half (A: top, B: bottom)
constexpr int kPR = kHalf + 4;      // packed key rows: input rows of one half
static_assert(kMR % 4 == 0 && kMC % 8 == 0, "median blocks are 2 x 8, two per thread");
static_assert((kHalf / 2) * (kMC / 8) == kThreadsB, "two median blocks per thread");
static_assert(kES % 4 == 0 && kEC % 4 == 0 && kTBW % 4 == 0, "16-byte rows and chunks");
static_assert(kER * kES >= kMR * kMS, "the median output as floats fits in the region buffer");

struct FloatOps {
    static __device__ __forceinline__ float min2(float a, float b) { return fminf(a, b); }
    static __device__ __forceinline__ float max2(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float min3(float a, float b, float c)
    {
        float r;
        asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
        return r;
    }
    static __device__ __forceinline__ float max3(float a, float b, float c)
    {
        float r;
        asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
        return r;
    }
};

// Two unsigned 16-bit keys per register.
struct PackedKeyOps {
    static __device__ __forceinline__ unsigned min2(unsigned a, unsigned b) { return __vminu2(a, b); }
    static __device__ __forceinline__ unsigned max2(unsigned a, unsigned b) { return __vmaxu2(a, b); }
    static __device__ __forceinline__ unsigned min3(unsigned a, unsigned b, unsigned c)
    {
        return __vimin3_u16x2(a, b, c);
    }
    static __device__ __forceinline__ unsigned max3(unsigned a, unsigned b, unsigned c)
    {
        return __vimax3_u16x2(a, b, c);
    }
};


__device__ __forceinline__ int clampi(int p, int n) { return p < 0 ? 0 : (p >= n ? n - 1 : p); }

// Mirror p into [0, n) without repeating the edge pixel (reflect-101).
__device__ __forceinline__ int reflect101(int p, int n)
{
    if (n == 1) return 0;
    while (p < 0 || p >= n) p = (p < 0) ? -p : 2 * (n - 1) - p;
    return p;
}

struct Tile {
    FrameDesc fd;
    int y0, x0;  // first output pixel
    int f;       // frame index in the batch
};

// Positions of a rows x cols region (origin at tile pixel - w) that lie
// outside the frame but within w of it: up to w rows above and below (all
// columns), and up to w columns left and right of the in-frame rows.
struct Ring {
    int top, bot0, bot1, left, right0, right1, cols, in0, in1;
    __device__ __forceinline__ int count() const
    {
        return (top + (bot1 - bot0)) * cols + (left + (right1 - right0)) * (in1 - in0);
    }
    __device__ __forceinline__ void at(int i, int& a, int& b) const
    {
        const int nr = (top + (bot1 - bot0)) * cols;
        if (i < nr) {
            const int r = i / cols;
            b = i - r * cols;
            a = r < top ? r : bot0 + (r - top);
        } else {
            i -= nr;
            const int span = in1 - in0;
            const int c = i / span;
            a = in0 + (i - c * span);
            b = c < left ? c : right0 + (c - left);
        }
    }
};

__device__ __forceinline__ Ring ring_of(const Tile& T, int w, int rows, int cols)
{
    Ring r;
    r.cols = cols;
    r.top = T.y0 < w ? w - T.y0 : 0;                 // region rows [0, top) are above the frame
    r.bot0 = min(T.fd.H - T.y0 + w, rows);           // first region row below the frame
    r.bot1 = min(r.bot0 + w, rows);
    r.left = T.x0 < w ? w - T.x0 : 0;
    r.right0 = min(T.fd.W - T.x0 + w, cols);
    r.right1 = min(r.right0 + w, cols);
    r.in0 = r.top;                                   // in-frame region rows
    r.in1 = r.bot0;
    return r;
}

// Tile t of the batch.  With frames of one shape (row_stride = the batch's
// tiles per tile row) tiles go by tile rows over the whole batch from the
// bottom up: the costly rows (data, empty pixels) are handed out first and
// the cheap ones above every column's top (one computed row) last, so the
// kernel's tail is short.  Otherwise frame by frame, row-major.
__device__ __forceinline__ Tile tile_of(const FrameDesc* __restrict__ frames, int n_frames, int t, int row_stride)
{
    Tile T;
    if (row_stride > 0) {
        const int r = t / row_stride, g = t - r * row_stride;
        const int f = g / frames[0].tiles_x_b;
        T.fd = frames[f];
        T.y0 = ((T.fd.H + kTBH - 1) / kTBH - 1 - r) * kTBH;
        T.x0 = (g - f * T.fd.tiles_x_b) * kTBW;
        T.f = f;
        return T;
    }
    const int f = find_frame<false>(frames, n_frames, t);
    T.fd = frames[f];
    T.f = f;
    const int local = t - T.fd.base_b;
    const int ty = local / T.fd.tiles_x_b;
    T.y0 = ty * kTBH;
    T.x0 = (local - ty * T.fd.tiles_x_b) * kTBW;
    return T;
}

// Column tops and the keys of their values for columns [xa, xa + n)
// (clamped into the frame), into ctop / ctv (kNoTop, 0: none, or step 5 off).
__device__ __forceinline__ void load_tops(const Tile& T, const StageBParams& p, int xa, int n,
                                          int* ctop, unsigned* ctv)
{
    for (int i = threadIdx.x; i < n; i += kThreadsB) {
        const int x = clampi(xa + i, T.fd.W);
        int top = kNoTop;
        unsigned k = 0u;
        if (p.extend_top) {
            const unsigned long long t = T.fd.top[x];  // row and key in one load
            if (t != kNoTopPacked) {
                top = (int)(t >> 32);
                k = (unsigned)t;
            }
        }
        ctop[i] = top;
        ctv[i] = k;
    }
}

// The top values of load_tops as floats, in place (ctv's words become the
// floats' bits): k / 256, or the float map's value for an off-grid one.
__device__ __forceinline__ void tops_to_floats(const Tile& T, int xa, int n, const int* ctop, unsigned* ctv)
{
    for (int i = threadIdx.x; i < n; i += kThreadsB) {
        const int top = ctop[i];
        const float v = top == kNoTop ? 0.0f : top_value(T.fd, top, ctv[i], clampi(xa + i, T.fd.W));
        ctv[i] = __float_as_uint(v);
    }
}

__device__ __forceinline__ bool above_top(const StageBParams& p, int y, int top)
{
    return (top != kNoTop) && y < top && (p.extend_rows < 0 || y >= top - p.extend_rows);
}

// E at frame pixel (y, x) (in frame), from C and the column's top.
__device__ __forceinline__ float extended(const Tile& T, const StageBParams& p, int y, int x,
                                          int top, float topval)
{
    return above_top(p, y, top) ? topval : c_at(T.fd, y, x);
}

// The same as a key (kKeyOff where C is off the key grid).
__device__ __forceinline__ unsigned extended_key(const Tile& T, const StageBParams& p, int y, int x,
                                                 int top, unsigned topkey)
{
    return above_top(p, y, top) ? topkey : (unsigned)T.fd.ck[(size_t)y * T.fd.c_pitch + x];
}

// Whether E (C after step 5) is empty in frame column x from row 0 to row
// `last`: C is empty above the column's top row (its first non-empty one),
// and step 5 writes nothing there when it is off or capped short of `last`.
// Reads the top itself: the tops of load_tops are cleared when step 5 is off.
__device__ __forceinline__ bool column_empty_to(const Tile& T, const StageBParams& p, int x, int last)
{
    const unsigned long long t = __ldg(T.fd.top + x);
    if (t == kNoTopPacked) return true;
    const int top = (int)(t >> 32);
    if (top <= last) return false;
    return !p.extend_top || (p.extend_rows >= 0 && last < top - p.extend_rows);
}

// The output of a tile whose median is empty everywhere: 0 (step 8 writes 0
// where the median is empty, whatever the blur).
__device__ void store_zero_tile(const Tile& T)
{
    for (int i = threadIdx.x; i < kTBH * kTBW; i += kThreadsB) {
        const int a = i / kTBW, b = i - a * kTBW;
        const int y = T.y0 + a, x = T.x0 + b;
        if (y < T.fd.H && x < T.fd.W) T.fd.out[(size_t)y * T.fd.out_pitch + x] = 0.0f;
    }
}

// The median output region M (kMR x kMS): 16-bit keys (Mk) after the packed
// median, floats (Mf) otherwise.  These read one value as a float.
template <bool KEYS>
__device__ __forceinline__ float m_at(const float* __restrict__ Mf, const unsigned short* __restrict__ Mk, int i)
{
    if constexpr (KEYS) return key_value(Mk[i]);
    else return Mf[i];
}

// Eight consecutive values of M from index i (a multiple of 4).
template <bool KEYS>
__device__ __forceinline__ void m_row8(const float* __restrict__ Mf, const unsigned short* __restrict__ Mk, int i,
                                       float (&v)[8])
{
    if constexpr (KEYS) {
        const uint2 lo = *reinterpret_cast<const uint2*>(Mk + i);
        const uint2 hi = *reinterpret_cast<const uint2*>(Mk + i + 4);
        const unsigned w[4] = {lo.x, lo.y, hi.x, hi.y};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[2 * j] = key_value(w[j] & 0xFFFFu);
            v[2 * j + 1] = key_value(w[j] >> 16);
        }
    } else {
        const float4 lo = *reinterpret_cast<const float4*>(Mf + i);
        const float4 hi = *reinterpret_cast<const float4*>(Mf + i + 4);
        v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
        v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
    }
}

// After the median: mirrored ring, blur, inversion, store.  R (kMR x kRS
// floats) is the Gaussian row-pass buffer; it must not overlap M.  On keys
// the Gaussian is exact: every median value is k / 256 with an integer k <=
// 25600 (inverted depths are below 100), so its binomial 5 x 5 sum is n /
// 2^16 with an integer n < 2^23, a float; step 8 then rounds 100 - n / 2^16
// once, as the exact definition does.
template <bool KEYS>
__device__ void blur_store(const Tile& T, const StageBParams& p, float* __restrict__ Mf,
                           unsigned short* __restrict__ Mk, float* __restrict__ R)
{
    const int H = T.fd.H, W = T.fd.W;
    const int tid = threadIdx.x;
    // -- mirror the ring outside the frame (the blur's reflect-101 border):
    // only the two rows / columns beyond each edge are read by the blur
    const bool edge = T.y0 < 2 || T.x0 < 2 || T.y0 + kTBH + 2 > H || T.x0 + kTBW + 2 > W;
    if (edge) {
        const Ring ring = ring_of(T, 2, kMR, kMC);
        for (int i = tid; i < ring.count(); i += kThreadsB) {
            int a, b;
            ring.at(i, a, b);
            const int y = T.y0 - 2 + a, x = T.x0 - 2 + b;
            if (y < -2 || y >= H + 2 || x < -2 || x >= W + 2) continue;
            const int sy = reflect101(y, H) - (T.y0 - 2), sx = reflect101(x, W) - (T.x0 - 2);
            if constexpr (KEYS) Mk[a * kMS + b] = Mk[sy * kMS + sx];
            else Mf[a * kMS + b] = Mf[sy * kMS + sx];
        }
        __syncthreads();
    }
    if (p.stop == kStopMedian) {
        for (int i = tid; i < kTBH * kTBW; i += kThreadsB) {
            const int a = i / kTBW, b = i - a * kTBW;
            const int y = T.y0 + a, x = T.x0 + b;
            if (y < H && x < W) T.fd.out[(size_t)y * T.fd.out_pitch + x] = m_at<KEYS>(Mf, Mk, (a + 2) * kMS + b + 2);
        }
        return;
    }
    constexpr float w0 = 0.0625f, w1 = 0.25f, w2 = 0.375f;  // [1 4 6 4 1] / 16
    if (p.blur == kBlurGauss) {
        // row pass over all kMR rows of M, the tile's kTBW columns -> R
        for (int i = tid; i < kMR * (kTBW / 4); i += kThreadsB) {
            const int a = i / (kTBW / 4), b0 = 4 * (i - a * (kTBW / 4));
            if constexpr (KEYS) {
                // the integer sums n = k(-2) + 4 k(-1) + 6 k + 4 k(1) + k(2) of the
                // keys in float arithmetic (exact: every value is an integer below
                // 2^24), stored as n + 1 with the sign of the centre's emptiness:
                // +(n + 1) when its key is not empty, -(n + 1) when it is.  A key
                // becomes a float as 2^23 + k (the key in the low bits) - 2^23.
                const uint2 lo = *reinterpret_cast<const uint2*>(Mk + a * kMS + b0);
                const uint2 hi = *reinterpret_cast<const uint2*>(Mk + a * kMS + b0 + 4);
                const unsigned w[4] = {lo.x, lo.y, hi.x, hi.y};
                float k[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    k[2 * j] = __uint_as_float(__byte_perm(w[j], 0x4B000000u, 0x7410)) - 8388608.0f;
                    k[2 * j + 1] = __uint_as_float(__byte_perm(w[j], 0x4B000000u, 0x7432)) - 8388608.0f;
                }
                float o[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float n1 = fmaf(6.0f, k[j + 2], fmaf(4.0f, k[j + 1] + k[j + 3], k[j] + k[j + 4])) + 1.0f;
                    // +1 when the centre's key is above kEmptyKeyMax (keys are integers), else -1
                    const float sgn = fmaf(2.0f, __saturatef(k[j + 2] - (float)kEmptyKeyMax), -1.0f);
                    o[j] = n1 * sgn;
                }
                *reinterpret_cast<float4*>(R + a * kRS + b0) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
                float v[8];
                m_row8<KEYS>(Mf, Mk, a * kMS + b0, v);
                float o[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float acc = w0 * v[k];
                    acc = fmaf(w1, v[k + 1], acc);
                    acc = fmaf(w2, v[k + 2], acc);
                    acc = fmaf(w1, v[k + 3], acc);
                    acc = fmaf(w0, v[k + 4], acc);
                    o[k] = acc;
                }
                *reinterpret_cast<float4*>(R + a * kRS + b0) = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
        __syncthreads();
    }
    if (p.blur == kBlurGauss) {
        // column pass, masked by the median, inverted, stored: each thread
        // takes kGRows rows of two adjacent columns
        constexpr int kPairs = kTBW / 2, kGRows = kTBH / 4;
        static_assert(kTBW % 2 == 0 && kTBH % 4 == 0 && kThreadsB >= 4 * kPairs && kRS % 2 == 0 && kMS % 2 == 0,
                      "column-pass mapping");
        if (tid < 4 * kPairs) {
            const int cp = tid % kPairs, a0 = (tid / kPairs) * kGRows;
            const int b = 2 * cp, x = T.x0 + b;
            const int rows = min(kGRows, H - (T.y0 + a0));
            if (x < W && rows > 0) {
                // a window of five row-pass rows, slid down the strip (on keys
                // five rows per round, so that no register moves; on floats and
                // for the blur stop a rolled loop: the kernel's code is large
                // and shares the instruction cache between five CTAs in
                // different phases)
                float2 r[5];
#pragma unroll
                for (int k = 0; k < 4; ++k) r[k] = *reinterpret_cast<const float2*>(R + (a0 + k) * kRS + b);
                const bool two = x + 1 < W;
                // both outputs in one 8-byte store when every row keeps them aligned
                const bool vec = two && (T.fd.out_pitch % 2) == 0 &&
                                 (reinterpret_cast<uintptr_t>(T.fd.out + x) % sizeof(float2)) == 0;
                float* dst = T.fd.out + (size_t)(T.y0 + a0) * T.fd.out_pitch + x;
                if constexpr (KEYS) {
                    if (p.stop != kStopBlur) {
                        // sum of the weights times |R| = n + 16 for the 5 x 5 integer sum
                        // n; 100 - n / 2^16 = c - (n + 16) / 2^16 rounded once (c = 100 +
                        // 2^-12 is a float), times 1 (centre not empty: R > 0) or 0.  All
                        // in float arithmetic; five rows per round so that the window
                        // slides through the registers without moves
                        constexpr float c = 100.0f + 16.0f / 65536.0f;
#pragma unroll 1
                        for (int k0 = 0; k0 < rows; k0 += 5) {
#pragma unroll
                            for (int u = 0; u < 5; ++u) {
                                const int k = k0 + u;
                                if (k < rows) {
                                    r[(u + 4) % 5] = *reinterpret_cast<const float2*>(R + (a0 + k + 4) * kRS + b);
                                    const float2 q0 = r[u % 5], q1 = r[(u + 1) % 5], q2 = r[(u + 2) % 5],
                                                 q3 = r[(u + 3) % 5], q4 = r[(u + 4) % 5];
                                    const float s0 = fmaf(6.0f, fabsf(q2.x),
                                                          fmaf(4.0f, fabsf(q1.x) + fabsf(q3.x), fabsf(q0.x) + fabsf(q4.x)));
                                    const float s1 = fmaf(6.0f, fabsf(q2.y),
                                                          fmaf(4.0f, fabsf(q1.y) + fabsf(q3.y), fabsf(q0.y) + fabsf(q4.y)));
                                    const float o0 = fmaf(-s0, 1.0f / 65536.0f, c) * __saturatef(q2.x);
                                    const float o1 = fmaf(-s1, 1.0f / 65536.0f, c) * __saturatef(q2.y);
                                    float* d = dst + (size_t)k * T.fd.out_pitch;
                                    if (vec) {
                                        *reinterpret_cast<float2*>(d) = make_float2(o0, o1);
                                    } else {
                                        d[0] = o0;
                                        if (two) d[1] = o1;
                                    }
                                }
                            }
                        }
                        return;
                    }
                }
#pragma unroll 1
                for (int k = 0; k < rows; ++k) {
                    r[4] = *reinterpret_cast<const float2*>(R + (a0 + k + 4) * kRS + b);
                    const int mi = (a0 + k + 2) * kMS + b + 2;
                    bool e0, e1;
                    if constexpr (KEYS) {
                        const unsigned w = *reinterpret_cast<const unsigned*>(Mk + mi);
                        e0 = (w & 0xFFFFu) <= kEmptyKeyMax;
                        e1 = (w >> 16) <= kEmptyKeyMax;
                    } else {
                        const float2 m2 = *reinterpret_cast<const float2*>(Mf + mi);
                        e0 = is_empty(m2.x);
                        e1 = is_empty(m2.y);
                    }
                    float acc0, acc1;
                    if constexpr (KEYS) {
                        // the blur n / 2^16 exactly (n < 256 * 25600 < 2^23): the sum of the
                        // weights times |R| is n + 16 (the row pass's +1s)
                        const float s0 = fmaf(6.0f, fabsf(r[2].x),
                                              fmaf(4.0f, fabsf(r[1].x) + fabsf(r[3].x), fabsf(r[0].x) + fabsf(r[4].x)));
                        const float s1 = fmaf(6.0f, fabsf(r[2].y),
                                              fmaf(4.0f, fabsf(r[1].y) + fabsf(r[3].y), fabsf(r[0].y) + fabsf(r[4].y)));
                        acc0 = fmaf(s0, 1.0f / 65536.0f, -16.0f / 65536.0f);
                        acc1 = fmaf(s1, 1.0f / 65536.0f, -16.0f / 65536.0f);
                    } else {
                        acc0 = w0 * r[0].x;
                        acc1 = w0 * r[0].y;
                        acc0 = fmaf(w1, r[1].x, acc0);
                        acc1 = fmaf(w1, r[1].y, acc1);
                        acc0 = fmaf(w2, r[2].x, acc0);
                        acc1 = fmaf(w2, r[2].y, acc1);
                        acc0 = fmaf(w1, r[3].x, acc0);
                        acc1 = fmaf(w1, r[3].y, acc1);
                        acc0 = fmaf(w0, r[4].x, acc0);
                        acc1 = fmaf(w0, r[4].y, acc1);
                    }
                    float o0, o1;
                    if (p.stop == kStopBlur) {  // the blurred map itself (inverted domain)
                        o0 = e0 ? m_at<KEYS>(Mf, Mk, mi) : acc0;
                        o1 = e1 ? m_at<KEYS>(Mf, Mk, mi + 1) : acc1;
                    } else {
                        o0 = e0 ? 0.0f : __fsub_rn(kInvertFrom, acc0);
                        o1 = e1 ? 0.0f : __fsub_rn(kInvertFrom, acc1);
                    }
                    if (vec) {
                        *reinterpret_cast<float2*>(dst) = make_float2(o0, o1);
                    } else {
                        dst[0] = o0;
                        if (two) dst[1] = o1;
                    }
                    dst += T.fd.out_pitch;
                    r[0] = r[1];
                    r[1] = r[2];
                    r[2] = r[3];
                    r[3] = r[4];
                }
            }
        }
        return;
    }
    // bilateral or no blur, masked by the median, inverted, stored: each
    // thread takes kStripRows rows of one column.  The bilateral reads the
    // median output as floats, converted from keys once (into R, free now)
    const float* Mv = Mf;
    if constexpr (KEYS) {
        if (p.blur == kBlurBilateral) {
            for (int i = tid; i < kMR * kMS; i += kThreadsB) R[i] = key_value(Mk[i]);
            __syncthreads();
            Mv = R;
        }
    }
    constexpr int kStrips = kThreadsB / 64;
    constexpr int kStripRows = kTBH / kStrips;
    static_assert(kTBW <= 64 && kTBH % kStrips == 0, "column-pass mapping");
    const int b = tid & 63, a0 = (tid >> 6) * kStripRows;
    const int x = T.x0 + b;
    if (b < kTBW && x < W) {
        for (int k = 0; k < kStripRows; ++k) {
            const int a = a0 + k, y = T.y0 + a;
            if (y >= H) break;
            const float m = m_at<KEYS>(Mf, Mk, (a + 2) * kMS + b + 2);
            float g = m;
            if (!is_empty(m) && p.blur == kBlurBilateral) {
                float num = 0.0f, den = 0.0f;
#pragma unroll
                for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
                    for (int dx = -2; dx <= 2; ++dx) {
                        const int r2 = dy * dy + dx * dx;
                        if (r2 > 4) continue;
                        const float v = Mv[(a + 2 + dy) * kMS + b + 2 + dx];
                        const float d = v - m;
                        // CUDA's fast exponential: its relative error (a few ulp for the
                        // weights that count) moves the blur by well under 1e-4 m
                        const float wgt = p.ws[r2] * __expf(-(d * d) * p.inv_2sc2);
                        num = fmaf(v, wgt, num);
                        den += wgt;
                    }
                g = num / den;
            }
            const float o = (p.stop == kStopBlur) ? g : (is_empty(m) ? 0.0f : __fsub_rn(kInvertFrom, g));
            T.fd.out[(size_t)y * T.fd.out_pitch + x] = o;
        }
    }
}

// Region position (k, l) from the packed keys K: rows k < kPR are the low
// halves of K row k, rows k >= kHalf the high halves of K row k - kHalf.
__device__ __forceinline__ unsigned key_at(const unsigned* K, int k, int l)
{
    const unsigned short* h = reinterpret_cast<const unsigned short*>(K);
    return k < kPR ? h[2 * (k * kES + l)] : h[2 * ((k - kHalf) * kES + l) + 1];
}

// The shared tail.  F: the median input (kER x kES floats, border
// replicated).  K: the same values as packed 16-bit keys (row k of the top
// half in the low halves of K row k, row k + kHalf in the high halves) when
// `keys` is set (F is then not read).  The median goes to Mk as 16-bit keys
// when it ran on keys, else to Mf as floats (Mf may alias K and Mk, which
// are then idle), then blur_store.  R (kMR x kRS floats) may alias F, not Mf
// or Mk.
__device__ void median_blur_store(const Tile& T, const StageBParams& p, const float* __restrict__ F,
                                  const unsigned* __restrict__ K, bool keys, float* __restrict__ Mf,
                                  unsigned short* __restrict__ Mk, float* __restrict__ R)
{
    const int tid = threadIdx.x;
    const bool use_keys = keys;
    // -- step 7: median, blocks (rb, cb) and (rb + kHalf / 2, cb) of 2 x 8
    const int rb = tid / (kMC / 8), cb = tid % (kMC / 8);
    if (!p.median && use_keys) {
        for (int i = tid; i < kMR * kMC; i += kThreadsB) {
            const int a = i / kMC, b = i - a * kMC;
            Mk[a * kMS + b] = (unsigned short)key_at(K, a + 2, b + 2);
        }
    } else if (!p.median) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int a = 2 * rb + h * kHalf + r, b = 8 * cb + j;
                    Mf[a * kMS + b] = F[(a + 2) * kES + b + 2];
                }
    } else if (use_keys) {
        unsigned x[6][12];
        const unsigned* src = K + (2 * rb) * kES + 8 * cb;
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const uint4 v = *reinterpret_cast<const uint4*>(src + r * kES + 4 * q);
                x[r][4 * q + 0] = v.x;
                x[r][4 * q + 1] = v.y;
                x[r][4 * q + 2] = v.z;
                x[r][4 * q + 3] = v.w;
            }
        unsigned m[2][8];
        median_block_2x8<unsigned, PackedKeyOps>(x, m);
        // low halves: the block in the top half, high halves: the bottom one
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const unsigned sel = h ? 0x7632u : 0x5410u;
                unsigned short* dst = Mk + (2 * rb + h * kHalf + r) * kMS + 8 * cb;
                *reinterpret_cast<uint4*>(dst) =
                    make_uint4(__byte_perm(m[r][0], m[r][1], sel), __byte_perm(m[r][2], m[r][3], sel),
                               __byte_perm(m[r][4], m[r][5], sel), __byte_perm(m[r][6], m[r][7], sel));
            }
    } else {
        // Mf may alias K and Mk: the float network reads only F
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float x[6][12];
            const float* src = F + (2 * rb + h * kHalf) * kES + 8 * cb;
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float4 v = *reinterpret_cast<const float4*>(src + r * kES + 4 * q);
                    x[r][4 * q + 0] = v.x;
                    x[r][4 * q + 1] = v.y;
                    x[r][4 * q + 2] = v.z;
                    x[r][4 * q + 3] = v.w;
                }
            float m[2][8];
            median_block_2x8<float, FloatOps>(x, m);
            float* dst = Mf + (2 * rb + h * kHalf) * kMS + 8 * cb;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                *reinterpret_cast<float4*>(dst + r * kMS) = make_float4(m[r][0], m[r][1], m[r][2], m[r][3]);
                *reinterpret_cast<float4*>(dst + r * kMS + 4) = make_float4(m[r][4], m[r][5], m[r][6], m[r][7]);
            }
        }
    }
    __syncthreads();
    if (use_keys) blur_store<true>(T, p, Mf, Mk, R);
    else blur_store<false>(T, p, Mf, Mk, R);
}

// Step 6 at one empty pixel (y, x): the maximum of E over the in-frame part
// of its (2 Rl + 1)^2 window, read from C with step 5 applied.  One warp per
// pixel, lane = column offset; returns the maximum in every lane.
__device__ float large_fill_at(const Tile& T, const StageBParams& p, int y, int x, int lane)
{
    const int Rl = p.large_radius, H = T.fd.H, W = T.fd.W;
    const int ylo = max(0, y - Rl), yhi = min(H - 1, y + Rl);
    float m = ninf();
    for (int dx0 = -Rl; dx0 <= Rl; dx0 += 32) {
        const int dx = dx0 + lane;
        const int xx = x + dx;
        if (dx <= Rl && xx >= 0 && xx < W) {
            int top = kNoTop;
            float tv = 0.0f;
            if (p.extend_top) {
                const unsigned long long t = T.fd.top[xx];
                if (t != kNoTopPacked) {
                    top = (int)(t >> 32);
                    tv = top_value(T.fd, top, (unsigned)t, xx);
                }
            }
#pragma unroll 4
            for (int yy = ylo; yy <= yhi; ++yy) m = fmaxf(m, extended(T, p, yy, xx, top, tv));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

// Capacity of the list of empty pixels a tile fills itself; a tile with
// more than StageBParams::sparse_fill_max (<= this) goes to the worklist.
constexpr int kMaxSparseFill = 160;

// Region work is split by column chunk of 4: kER rows x kChunksPerRow.
constexpr int kChunksPerRow = kEC / 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The region's keys arrive as a kKeyBoxH x kKeyBoxW box Ek (16-bit, dense
// rows) whose first column is the region's first column x0 - 4 rounded down
// to a multiple of 8 (16 bytes): region column l is box column l + ko, ko 0
// or 4.  By one tensor copy (TMA): thread 0 arms the CTA's mbarrier with the
// byte count and starts the copy of the box at (x, y, frame) of C's keys;
// parts outside the frame arrive as zeros.  Every thread then waits for the
// barrier's phase, a bounded number of times.
static_assert(kKeyBoxW == kEC + 4 && kKeyBoxH == kER && (kKeyBoxW * 2) % 16 == 0, "the key box");
static_assert(kKeyBoxW * kKeyBoxH * 2 <= kER * kES * 4, "the key box fits in the region buffer");
constexpr unsigned kRegionBytes = kKeyBoxW * kKeyBoxH * 2;
__device__ __forceinline__ int key_box_x(int x0) { return (x0 - 4) & ~7; }

__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void tma_region(float* dst, const CUtensorMap* map, int x, int y, int f,
                                           unsigned long long* mbar)
{
    // earlier reads and writes of dst (the previous tile) before the copy writes it
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mbar)),
                 "r"(kRegionBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(f), "r"(smem_addr(mbar))
        : "memory");
}

// Wait until the barrier's current phase (parity) completes; false if it
// has not after ~4M polls (each poll may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait(unsigned long long* mbar, unsigned parity)
{
    const unsigned a = smem_addr(mbar);
    for (int i = 0; i < (1 << 22); ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Region work is split by column chunk: thread t < kRowGroups x kChunksPerRow
// takes chunk t % kChunksPerRow of every kRowGroups-th row from t /
// kChunksPerRow, so its column bounds and column tops are computed once.
constexpr int kRowGroups = kThreadsB / kChunksPerRow;

// Start copying a tile's key box into `dst` by 16-byte cp.async chunks of 8
// keys: the in-frame ones (rows of C's keys are padded to 32 keys, so a chunk
// straddling the right edge reads allocated padding; key_box_x is a multiple
// of 8, so no chunk straddles the left edge).  The rest is left as it was.
__device__ __forceinline__ void issue_region_keys(const Tile& T, unsigned short* dst)
{
    constexpr int kChunks = kKeyBoxW / 8;
    const int xb = key_box_x(T.x0);
    for (int i = threadIdx.x; i < kKeyBoxH * kChunks; i += kThreadsB) {
        const int k = i / kChunks, j = i - k * kChunks;
        const int y = T.y0 - 4 + k, x = xb + 8 * j;
        if (y >= 0 && y < T.fd.H && x >= 0 && x < T.fd.W)
            cp_async16(dst + k * kKeyBoxW + 8 * j, T.fd.ck + (size_t)y * T.fd.c_pitch + x);
    }
    cp_async_commit();
}

// Write the key of region position (k, l) into K's half-words.
__device__ __forceinline__ void put_key(unsigned* K, int k, int l, unsigned key)
{
    unsigned short* h = reinterpret_cast<unsigned short*>(K);
    if (k < kPR) h[2 * (k * kES + l)] = static_cast<unsigned short>(key);
    if (k >= kHalf) h[2 * ((k - kHalf) * kES + l) + 1] = static_cast<unsigned short>(key);
}

// Keys of the whole region from E (after step 6 on a tile whose scratch
// took K): the same values the fix pass writes, pairs of rows (kp, kp + kHalf).
__device__ void build_keys(const Tile& T, const float* __restrict__ E, unsigned* __restrict__ K, bool& ok)
{
    const int H = T.fd.H, W = T.fd.W;
    for (int i = threadIdx.x; i < kPR * kChunksPerRow; i += kThreadsB) {
        const int kp = i / kChunksPerRow, q = i - kp * kChunksPerRow;
        const int xs = T.x0 - 4 + 4 * q;
        unsigned key[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = kp + h * kHalf;
            const int y = T.y0 - 4 + k;
            if (y < 0 || y >= H || xs < 0 || xs >= W) continue;
            const float4 c4 = *reinterpret_cast<const float4*>(E + k * kES + 4 * q);
            const float v[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (xs + e >= W) break;
                key[h][e] = key_of(v[e], ok);
            }
        }
        *reinterpret_cast<uint4*>(K + kp * kES + 4 * q) =
            make_uint4(key[0][0] | (key[1][0] << 16), key[0][1] | (key[1][1] << 16),
                       key[0][2] | (key[1][2] << 16), key[0][3] | (key[1][3] << 16));
    }
}

// A tile whose whole region lies above its columns' top rows (step 5 then
// makes every row of the region the same: E(y, x) = C(top(x), x)) has
// row-constant maps: the median of a window is the median of its five column
// values (each appears five times), and the blur sums identical rows.  This
// computes one output row with the same operations, in the same order, as
// the general path, and writes it to every row of the tile.  cval holds the
// region's top values (border replicated); W (kMC + kTBW floats) is scratch.
__device__ void constant_tile_store(const Tile& T, const StageBParams& p, const float* __restrict__ cval,
                                    float* __restrict__ W_)
{
    const int H = T.fd.H, W = T.fd.W;
    const int tid = threadIdx.x;
    float* Mrow = W_;          // kMC: median region columns
    float* Orow = W_ + kMC;    // kTBW: the output row
    float m = 0.0f;
    if (tid < kMC) {
        float v[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = cval[tid + j];
        if (p.median) {
#pragma unroll
            for (int i = 1; i < 5; ++i)
#pragma unroll
                for (int j = 4; j >= i; --j) {
                    const float lo = fminf(v[j - 1], v[j]), hi = fmaxf(v[j - 1], v[j]);
                    v[j - 1] = lo;
                    v[j] = hi;
                }
        }
        m = v[2];
        Mrow[tid] = m;
    }
    __syncthreads();
    // reflect-101 of the two columns beyond each frame edge
    if (tid < kMC) {
        const int x = T.x0 - 2 + tid;
        if ((x < 0 || x >= W) && x >= -2 && x < W + 2) m = Mrow[reflect101(x, W) - (T.x0 - 2)];
    }
    __syncthreads();
    if (tid < kMC) Mrow[tid] = m;
    // all of them 16-bit keys: the blur below is exact, as in the general path
    bool ok = true;
    if (tid < kMC) key_of(m, ok);
    const bool keys = __syncthreads_and(ok);
    constexpr float w0 = 0.0625f, w1 = 0.25f, w2 = 0.375f;
    if (tid < kTBW) {
        const int b = tid;
        const float mc = Mrow[b + 2];
        float o = mc;
        if (p.stop == kStopExtend || p.stop == kStopFillLarge) {
            o = cval[b + 4];
        } else if (p.stop != kStopMedian) {
            float g = mc;
            if (!is_empty(mc)) {
                if (p.blur == kBlurGauss && keys) {
                    // the 5 x 5 sum over keys is 16 times the row sum n over keys:
                    // the blur is n / 2^12 (n < 16 * 25600 < 2^23)
                    bool unused = true;
                    unsigned kk[5];
#pragma unroll
                    for (int j = 0; j < 5; ++j) kk[j] = key_of(Mrow[b + j], unused);
                    const unsigned n = kk[0] + kk[4] + 4u * (kk[1] + kk[3]) + 6u * kk[2];
                    g = __uint_as_float(0x45000000u | n) - 2048.0f;
                } else if (p.blur == kBlurGauss) {
                    float r = w0 * Mrow[b];
                    r = fmaf(w1, Mrow[b + 1], r);
                    r = fmaf(w2, Mrow[b + 2], r);
                    r = fmaf(w1, Mrow[b + 3], r);
                    r = fmaf(w0, Mrow[b + 4], r);
                    float acc = w0 * r;
                    acc = fmaf(w1, r, acc);
                    acc = fmaf(w2, r, acc);
                    acc = fmaf(w1, r, acc);
                    acc = fmaf(w0, r, acc);
                    g = acc;
                } else if (p.blur == kBlurBilateral) {
                    float num = 0.0f, den = 0.0f;
#pragma unroll
                    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
                        for (int dx = -2; dx <= 2; ++dx) {
                            const int r2 = dy * dy + dx * dx;
                            if (r2 > 4) continue;
                            const float v = Mrow[b + 2 + dx];
                            const float d = v - mc;
                            const float wgt = p.ws[r2] * __expf(-(d * d) * p.inv_2sc2);  // as in blur_store
                            num = fmaf(v, wgt, num);
                            den += wgt;
                        }
                    g = num / den;
                }
            }
            o = (p.stop == kStopBlur) ? g : (is_empty(mc) ? 0.0f : __fsub_rn(kInvertFrom, g));
        }
        Orow[b] = o;
    }
    __syncthreads();
    // every row the same: thread (half, column) writes half a column
    static_assert(kThreadsB == 128 && kTBW <= 64 && kTBH % 2 == 0, "two threads per column");
    const int b = tid & 63, a0 = (tid >> 6) * (kTBH / 2);
    const int x = T.x0 + b;
    if (b < kTBW && x < W) {
        const float o = Orow[b];
        float* dst = T.fd.out + (size_t)(T.y0 + a0) * T.fd.out_pitch + x;
        const int rows = min(kTBH / 2, H - (T.y0 + a0));
        for (int a = 0; a < rows; ++a, dst += T.fd.out_pitch) *dst = o;
    }
}

// Shared memory of phase 1: the region (its key box on the key path, E as
// floats on the float path; the Gaussian's row-pass buffer after the
// median), the packed keys K, the median output as 16-bit keys Mk (the float
// median output Mf lies over K and Mk, which are idle on that path), extra
// step-6 scratch X, column tops, the empty pixels (list, and their columns
// as a bitmap, a list and an index).  Before the median, Mk and X are step-6
// scratch (kSmallScratch floats); on the float path a tile that needs more
// also takes K and rebuilds its keys afterwards (kBigScratch floats), on the
// key path the region buffer is free once K holds the keys.  The total
// leaves room for five CTAs per SM (233,472 bytes; allocations in 128-byte
// units, 1 KB reserved per CTA).
constexpr int kScratchExtra = 1792;
constexpr int kSmallScratch = kMR * kMS / 2 + kScratchExtra;
constexpr int kBigScratch = kPR * kES + kSmallScratch;
constexpr size_t kMainSmemFloats =
    kER * kES + kPR * kES + kMR * kMS / 2 + kScratchExtra + 2 * kEC + kMaxSparseFill + 4 + 4 + 2 * kEC;
constexpr size_t kMainStaticSmem = 128;  // s_next, ebox, the mbarrier: padded to the dynamic part's alignment
static_assert(kPR * kES + kMR * kMS / 2 >= kMR * kMS, "the float median output fits over K and Mk");
static_assert((kER * kES) % 4 == 0 && (kPR * kES) % 4 == 0 && kMS % 8 == 0, "16-byte aligned buffers and rows");
static_assert(5 * ((kMainSmemFloats * 4 + kMainStaticSmem + 127) / 128 * 128 + 1024) <= 233472,
              "five CTAs per SM");

// The CTA's buffers of phase 1.
struct MainSmem {
    float* E;            // the region: key box (key path), floats (float path); later the row-pass buffer
    unsigned* K;         // the region as packed keys
    unsigned short* Mk;  // median output, keys
    float* Mf;           // median output, floats (over K and Mk)
    float* scratch;      // kSmallScratch floats (Mk and X), idle until the median
    int* ctop;           // the region's column tops
    unsigned* ctv;       // their keys; their values' bits after tops_to_floats
    int* elist;          // empty pixels, (region row << 16) | region column
    int* ecount;
    unsigned* ecols;     // bitmap of region columns with empty pixels
    int* ecol_list;      // those columns, in order
    int* ecol_idx;       // region column -> position in the list
    int* ebox;           // region rows spanned by the empty pixels: kmin, kmax
};

__device__ __forceinline__ void reset_empties(const MainSmem& S)
{
    if (threadIdx.x == 0) {
        *S.ecount = 0;
        S.ebox[0] = 1 << 20;
        S.ebox[1] = -1;
        S.ecols[0] = S.ecols[1] = S.ecols[2] = 0u;
    }
}

// Record the empty pixels `em` (bit e: column 4 q + e) of region row k.
__device__ __forceinline__ void note_empties(const MainSmem& S, int k, int q, unsigned em)
{
    int slot = atomicAdd(S.ecount, __popc(em));
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if ((em >> e) & 1u) {
            if (slot < kMaxSparseFill) S.elist[slot] = (k << 16) | (4 * q + e);
            ++slot;
        }
    atomicMin(S.ebox + 0, k);
    atomicMax(S.ebox + 1, k);
    atomicOr(S.ecols + ((4 * q) >> 5), em << ((4 * q) & 31));
}

// The output of a tile from K (a stop after step 5 or 6: the map itself).
__device__ void store_keys_tile(const Tile& T, const unsigned* K)
{
    for (int i = threadIdx.x; i < kTBH * kTBW; i += kThreadsB) {
        const int a = i / kTBW, b = i - a * kTBW;
        const int y = T.y0 + a, x = T.x0 + b;
        if (y < T.fd.H && x < T.fd.W) T.fd.out[(size_t)y * T.fd.out_pitch + x] = key_value(key_at(K, a + 4, b + 4));
    }
}

// Step 6 at one empty pixel (y, x) on keys: the maximum key of E over the
// in-frame part of its window, from C's keys with step 5 applied; one warp
// per pixel, lane = column offset, the maximum in every lane.  `bad` is set
// when the window holds a value off the key grid (kKeyOff is the largest key).
__device__ unsigned large_fill_key_at(const Tile& T, const StageBParams& p, int y, int x, int lane, bool& bad)
{
    const int Rl = p.large_radius, H = T.fd.H, W = T.fd.W;
    const int ylo = max(0, y - Rl), yhi = min(H - 1, y + Rl);
    unsigned m = 0u;
    for (int dx0 = -Rl; dx0 <= Rl; dx0 += 32) {
        const int dx = dx0 + lane;
        const int xx = x + dx;
        if (dx <= Rl && xx >= 0 && xx < W) {
            int top = kNoTop;
            unsigned tk = 0u;
            if (p.extend_top) {
                const unsigned long long t = T.fd.top[xx];
                if (t != kNoTopPacked) {
                    top = (int)(t >> 32);
                    tk = (unsigned)t;
                }
            }
#pragma unroll 4
            for (int yy = ylo; yy <= yhi; ++yy) m = max(m, extended_key(T, p, yy, xx, top, tk));
        }
    }
    bad = bad || m > kKeyMax;
    return __reduce_max_sync(0xffffffffu, m);
}

// The empty pixels' distinct columns as a list (ecol_list, in order; ecol_idx
// maps a region column to its position), their number and the first and
// last.  Warps 0-2 take the bitmap's words.
__device__ __forceinline__ void empty_columns(const MainSmem& S, int& ND, int& lmin, int& lmax)
{
    const int tid = threadIdx.x;
    const unsigned w0 = S.ecols[0], w1 = S.ecols[1], w2 = S.ecols[2];
    if (tid < 96) {
        const int w = tid >> 5, lane = tid & 31;
        const unsigned bits = w == 0 ? w0 : (w == 1 ? w1 : w2);
        const int pos = (w > 0 ? __popc(w0) : 0) + (w > 1 ? __popc(w1) : 0) + __popc(bits & ((1u << lane) - 1u));
        if ((bits >> lane) & 1u) {
            S.ecol_list[pos] = tid;
            S.ecol_idx[tid] = pos;
        }
    }
    ND = __popc(w0) + __popc(w1) + __popc(w2);
    lmin = w0 ? __ffs(w0) - 1 : (w1 ? 31 + __ffs(w1) : 63 + __ffs(w2));
    lmax = w2 ? 95 - __clz(w2) : (w1 ? 63 - __clz(w1) : 31 - __clz(w0));
}

// Step 6 at the few empty pixels of a tile on keys (K holds the region with
// step 5 applied): the union of their windows (box) streams in row bands
// through the region buffer, idle now, keeping row maxima at their distinct
// columns in the scratch, then column maxima at each pixel; or, when that
// does not fit, one warp per pixel reading its window from C.  Writes the
// fills into K.  False (block-uniform) when a value read is off the key grid.
__device__ bool fill_keys(const Tile& T, const StageBParams& p, const MainSmem& S, int n_empty)
{
    const int tid = threadIdx.x, H = T.fd.H, W = T.fd.W, Rl = p.large_radius;
    int ND, lmin, lmax;
    empty_columns(S, ND, lmin, lmax);
    const int by0 = max(0, T.y0 - 4 + S.ebox[0] - Rl), by1 = min(H - 1, T.y0 - 4 + S.ebox[1] + Rl);
    const int bx0 = max(0, T.x0 - 4 + lmin - Rl), bx1 = min(W - 1, T.x0 - 4 + lmax + Rl);
    const int BR = by1 - by0 + 1, BC = bx1 - bx0 + 1;
    constexpr int kBandWords = kER * kES;
    bool bad = false;
    if (BR * ND <= kSmallScratch && 3 * BC <= kBandWords) {
        unsigned* rmax = reinterpret_cast<unsigned*>(S.scratch);
        int* btop = reinterpret_cast<int*>(S.E);
        unsigned* btk = reinterpret_cast<unsigned*>(btop + BC);
        unsigned* band = btk + BC;
        const int RB = min(BR, (kBandWords - 2 * BC) / BC);
        for (int c = tid; c < BC; c += kThreadsB) {
            int top = kNoTop;
            unsigned tk = 0u;
            if (p.extend_top) {
                const unsigned long long t2 = __ldg(T.fd.top + bx0 + c);
                if (t2 != kNoTopPacked) {
                    top = (int)(t2 >> 32);
                    tk = (unsigned)t2;
                }
            }
            btop[c] = top;
            btk[c] = tk;
        }
        __syncthreads();
        for (int r0 = 0; r0 < BR; r0 += RB) {
            const int nb = min(RB, BR - r0);
            // the band of E: inside the tile's region from K, elsewhere from C
            for (int i = tid; i < nb * BC; i += kThreadsB) {
                const int r = i / BC, c = i - r * BC;
                const int k = by0 + r0 + r - (T.y0 - 4), l = bx0 + c - (T.x0 - 4);
                unsigned v;
                if ((unsigned)k < (unsigned)kER && (unsigned)l < (unsigned)kEC) {
                    v = key_at(S.K, k, l);
                } else {
                    v = extended_key(T, p, by0 + r0 + r, bx0 + c, btop[c], btk[c]);
                    bad = bad || v > kKeyMax;
                }
                band[i] = v;
            }
            __syncthreads();
            // its row maxima over the window width at the empty columns
            for (int i = tid; i < nb * ND; i += kThreadsB) {
                const int r = i / ND, j = i - r * ND;
                const int c = T.x0 - 4 + S.ecol_list[j];
                const int lo = max(c - Rl, bx0) - bx0, hi = min(c + Rl, bx1) - bx0;
                unsigned m = 0u;
                for (int x = lo; x <= hi; ++x) m = max(m, band[r * BC + x]);
                rmax[(r0 + r) * ND + j] = m;
            }
            __syncthreads();
        }
        // column maxima at each empty pixel
        for (int j = tid; j < n_empty; j += kThreadsB) {
            const int k = S.elist[j] >> 16, l = S.elist[j] & 0xFFFF;
            const int y = T.y0 - 4 + k;
            const int lo = max(y - Rl, by0) - by0, hi = min(y + Rl, by1) - by0;
            const int jc = S.ecol_idx[l];
            unsigned m = 0u;
            for (int r = lo; r <= hi; ++r) m = max(m, rmax[r * ND + jc]);
            put_key(S.K, k, l, m);
        }
    } else {
        const int warp = tid >> 5, lane = tid & 31;
        for (int j = warp; j < n_empty; j += kThreadsB / 32) {
            const int k = S.elist[j] >> 16, l = S.elist[j] & 0xFFFF;
            const unsigned m = large_fill_key_at(T, p, T.y0 - 4 + k, T.x0 - 4 + l, lane, bad);
            if (lane == 0) put_key(S.K, k, l, m);
        }
    }
    return !__syncthreads_or(bad);
}

// A tile of the step-6 worklist, start to end (defined with its kernel).
__device__ void fill_tile_keys(const Tile& T, int t, const StageBParams& p, unsigned char* __restrict__ dynk,
                               int* __restrict__ ffill);

// Steps 5-8 of one tile on keys, from the key box in S.E (region column l
// at box column l + ko).  The fix pass moves the box into K: row pairs
// (kp, kp + kHalf) of one column chunk per thread, two 8-byte loads and four
// byte permutes per chunk, out-of-frame positions zeroed, step 5 applied
// from the column tops, empty pixels recorded (step 6).  Returns false,
// having stored nothing, when a value the tile needs is off the key grid.
// kInline: a tile with more empty pixels than it fills by itself runs the
// step-6 worklist's code at once, else it goes to the worklist.
template <bool kFill, bool kInline>
__device__ bool tile_keys(const Tile& T, const StageBParams& p, const MainSmem& S, int t, int* worklist,
                          int* ffill, bool ext_tile)
{
    const int tid = threadIdx.x, H = T.fd.H, W = T.fd.W;
    const unsigned short* Ek = reinterpret_cast<const unsigned short*>(S.E);
    unsigned* K = S.K;
    const int ko = (T.x0 - 4) - key_box_x(T.x0);
    unsigned mx = 0u;  // packed maximum of the keys this thread moved
    if (tid < kRowGroups * kChunksPerRow) {
        const int g = tid / kChunksPerRow, q = tid - g * kChunksPerRow;
        const int xs = T.x0 - 4 + 4 * q;
        const int ncol = (xs >= 0 && xs < W) ? min(4, W - xs) : 0;  // in-frame columns of the chunk
        const unsigned m0 = (ncol > 0 ? 0xFFFFu : 0u) | (ncol > 1 ? 0xFFFF0000u : 0u);
        const unsigned m1 = (ncol > 2 ? 0xFFFFu : 0u) | (ncol > 3 ? 0xFFFF0000u : 0u);
        const int klo = max(0, 4 - T.y0), khi = min(kER, H - T.y0 + 4);  // in-frame region rows
        // step 5 per column: region rows [elo, elo + espan) (the rows above
        // the top within the cap, inside the frame) take the top's key
        int elo[4];
        unsigned espan[4], ck[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int top = ext_tile ? S.ctop[4 * q + e] : kNoTop;
            const int hi = top == kNoTop ? 0 : min(khi, top - (T.y0 - 4));
            const int lo = max(klo, (top == kNoTop || p.extend_rows < 0) ? 0 : top - p.extend_rows - (T.y0 - 4));
            elo[e] = lo;
            espan[e] = (e < ncol && hi > lo) ? (unsigned)(hi - lo) : 0u;
            ck[e] = S.ctv[4 * q + e];
        }
        const unsigned short* src = Ek + ko + 4 * q;
        for (int kp = g; kp < kPR; kp += kRowGroups) {
            const int kb = kp + kHalf;
            uint2 a = *reinterpret_cast<const uint2*>(src + kp * kKeyBoxW);
            uint2 b = *reinterpret_cast<const uint2*>(src + kb * kKeyBoxW);
            const bool ina = kp >= klo && kp < khi, inb = kb >= klo && kb < khi;
            // chunks wholly inside the frame (nearly all) need no masks
            const bool inside = ncol == 4 && ina && inb;
            const unsigned ma0 = ina ? m0 : 0u, ma1 = ina ? m1 : 0u;
            const unsigned mb0 = inb ? m0 : 0u, mb1 = inb ? m1 : 0u;
            if (!inside) {
                a.x &= ma0;
                a.y &= ma1;
                b.x &= mb0;
                b.y &= mb1;
            }
            if (ext_tile) {  // step 5: a position above its column's top takes the top's key
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const unsigned sh = (e & 1) * 16, hm = 0xFFFFu << sh, kv = ck[e] << sh;
                    unsigned& wa = e < 2 ? a.x : a.y;
                    unsigned& wb = e < 2 ? b.x : b.y;
                    if ((unsigned)(kp - elo[e]) < espan[e]) wa = (wa & ~hm) | kv;
                    if ((unsigned)(kb - elo[e]) < espan[e]) wb = (wb & ~hm) | kv;
                }
            }
            mx = __vimax3_u16x2(mx, a.x, a.y);
            mx = __vimax3_u16x2(mx, b.x, b.y);
            if (kFill) {
                // empty in-frame positions (key <= kEmptyKeyMax); out-of-frame ones
                // are lifted out of the way.  Most chunks hold none: their
                // smallest key tells (adding 0x8000 - 26 to a half sets its top
                // bit exactly when its key is not empty; keys are below 0x8000)
                unsigned la0 = a.x, la1 = a.y, lb0 = b.x, lb1 = b.y;
                if (!inside) {
                    la0 |= ~ma0;
                    la1 |= ~ma1;
                    lb0 |= ~mb0;
                    lb1 |= ~mb1;
                }
                const unsigned mn = __vminu2(__vimin3_u16x2(la0, la1, lb0), lb1);
                if (((__vminu2(mn, 0x7FFF7FFFu) + 0x7FE67FE6u) & 0x80008000u) != 0x80008000u) {
                    unsigned ea = 0u, eb = 0u;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const unsigned sh = (e & 1) * 16;
                        ea |= ((((e < 2 ? la0 : la1) >> sh) & 0xFFFFu) <= kEmptyKeyMax ? 1u : 0u) << e;
                        eb |= ((((e < 2 ? lb0 : lb1) >> sh) & 0xFFFFu) <= kEmptyKeyMax ? 1u : 0u) << e;
                    }
                    // rows kHalf .. kPR - 1 appear in both halves: count them once
                    if (ea) note_empties(S, kp, q, ea);
                    if (eb && kp >= kPR - kHalf) note_empties(S, kb, q, eb);
                }
            }
            *reinterpret_cast<uint4*>(K + kp * kES + 4 * q) =
                make_uint4(__byte_perm(a.x, b.x, 0x5410), __byte_perm(a.x, b.x, 0x7632),
                           __byte_perm(a.y, b.y, 0x5410), __byte_perm(a.y, b.y, 0x7632));
        }
    }
    if (__syncthreads_or((mx & 0xFFFFu) > kKeyMax || (mx >> 16) > kKeyMax)) return false;
    const int n_empty = kFill ? *S.ecount : 0;  // no empties are counted without step 6
    if (p.stop == kStopExtend) {
        store_keys_tile(T, K);
        return true;
    }
    if (n_empty > T.fd.sparse_fill) {
        if constexpr (kInline) {  // the worklist tile's wide region fits here: do it now
            __syncthreads();      // every thread is done with this tile's buffers
            fill_tile_keys(T, t, p, reinterpret_cast<unsigned char*>(S.E), ffill);
        } else if (tid == 0) {
            const int slot = atomicAdd(worklist, 1);
            worklist[3 + slot] = t;
        }
        return true;
    }
    if (n_empty > 0 && !fill_keys(T, p, S, n_empty)) return false;
    // replicate the frame border into the two rows / columns beyond each
    // edge (the median's rule; farther ones feed only mirrored outputs)
    if (T.y0 < 2 || T.x0 < 2 || T.y0 + kTBH + 2 > H || T.x0 + kTBW + 2 > W) {
        const Ring ring = ring_of(T, 4, kER, kEC);
        for (int i = tid; i < ring.count(); i += kThreadsB) {
            int k, l;
            ring.at(i, k, l);
            const int y = T.y0 - 4 + k, x = T.x0 - 4 + l;
            if (y < -2 || y >= H + 2 || x < -2 || x >= W + 2) continue;
            put_key(K, k, l, key_at(K, clampi(y, H) - (T.y0 - 4), clampi(x, W) - (T.x0 - 4)));
        }
    }
    __syncthreads();
    if (p.stop == kStopFillLarge) store_keys_tile(T, K);
    else median_blur_store(T, p, nullptr, K, true, S.Mf, S.Mk, S.E);
    return true;
}

// Steps 5-8 of one tile on floats, for a tile with some value off the key
// grid: E from C's keys and the float map, then the same steps on floats
// (the median and blur still run on keys when the region's values allow).
template <bool kFill>
__device__ void tile_floats(const Tile& T, const StageBParams& p, const MainSmem& S, int t, int* ffill,
                            bool ext_tile)
{
    const int tid = threadIdx.x, H = T.fd.H, W = T.fd.W;
    float* E = S.E;
    unsigned* K = S.K;
    unsigned short* Mk = S.Mk;
    float* Mf = S.Mf;
    float* scratch = S.scratch;
    const int* ctop = S.ctop;
    int* elist = S.elist;
    int* ecount = S.ecount;
    unsigned* ecols = S.ecols;
    int* ecol_list = S.ecol_list;
    int* ecol_idx = S.ecol_idx;
    int* ebox = S.ebox;
    __syncthreads();  // the key path is done with every buffer
    reset_empties(S);
    tops_to_floats(T, T.x0 - 4, kEC, S.ctop, S.ctv);
    const float* cval = reinterpret_cast<const float*>(S.ctv);
    for (int i = tid; i < kER * kEC; i += kThreadsB) {
        const int k = i / kEC, l = i - k * kEC;
        const int y = T.y0 - 4 + k, x = T.x0 - 4 + l;
        if (y >= 0 && y < H && x >= 0 && x < W) E[k * kES + l] = c_at(T.fd, y, x);
    }
    __syncthreads();
    // step 5 in place, empty pixels, packed keys: row pairs (kp, kp + kHalf)
    // of one column chunk per thread
    bool keys_ok = true;
    if (tid < kRowGroups * kChunksPerRow) {
        const int g = tid / kChunksPerRow, q = tid - g * kChunksPerRow;
        const int xs = T.x0 - 4 + 4 * q;
        const int ncol = (xs >= 0 && xs < W) ? min(4, W - xs) : 0;  // in-frame columns of the chunk
        int ct[4];
        float cv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ct[e] = ext_tile ? ctop[4 * q + e] : kNoTop;
            cv[e] = ext_tile ? cval[4 * q + e] : 0.0f;
        }
        for (int kp = g; kp < kPR; kp += kRowGroups) {
            unsigned key[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = kp + h * kHalf;
                const int y = T.y0 - 4 + k;
                if (ncol == 0 || y < 0 || y >= H) continue;
                float4* cell = reinterpret_cast<float4*>(E + k * kES + 4 * q);
                const float4 c4 = *cell;
                float v[4] = {c4.x, c4.y, c4.z, c4.w};
                if (ext_tile) {
                    bool moved = false;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (above_top(p, y, ct[e])) {
                            v[e] = cv[e];
                            moved = true;
                        }
                    if (moved) *cell = make_float4(v[0], v[1], v[2], v[3]);
                }
                unsigned em = 0u;  // empty in-frame columns of this chunk row
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e < ncol) key[h][e] = key_of(v[e], keys_ok);
                // most chunks hold no empty pixel: test their smallest value first
                // (out-of-frame columns of a chunk at the right edge hold pixels
                // of the next row's start or padding, and are masked below)
                if (is_empty(fminf(fminf(v[0], v[1]), fminf(v[2], v[3]))))
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (e < ncol) em |= (is_empty(v[e]) ? 1u : 0u) << e;
                // rows kHalf .. kPR - 1 appear in both halves: count them once
                const bool counted = (h == 0) || (kp >= kPR - kHalf);
                if (em && counted && kFill) {
                    const int slot0 = atomicAdd(ecount, __popc(em));
                    int slot = slot0;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if ((em >> e) & 1u) {
                            if (slot < kMaxSparseFill) elist[slot] = (k << 16) | (4 * q + e);
                            ++slot;
                        }
                    atomicMin(ebox + 0, k);
                    atomicMax(ebox + 1, k);
                    atomicOr(ecols + ((4 * q) >> 5), em << ((4 * q) & 31));
                }
            }
            *reinterpret_cast<uint4*>(K + kp * kES + 4 * q) =
                make_uint4(key[0][0] | (key[1][0] << 16), key[0][1] | (key[1][1] << 16),
                           key[0][2] | (key[1][2] << 16), key[0][3] | (key[1][3] << 16));
        }
    }
    __syncthreads();
    const int n_empty = kFill ? *ecount : 0;  // no empties are counted without step 6

    auto store_tile = [&](const float* buf) {
        for (int i = tid; i < kTBH * kTBW; i += kThreadsB) {
            const int a = i / kTBW, b = i - a * kTBW;
            const int y = T.y0 + a, x = T.x0 + b;
            if (y < H && x < W) T.fd.out[(size_t)y * T.fd.out_pitch + x] = buf[(a + 4) * kES + b + 4];
        }
    };
    if (p.stop == kStopExtend) {
        store_tile(E);
    } else if (n_empty > T.fd.sparse_fill) {
        if (tid == 0) {
            const int slot = atomicAdd(ffill, 1);
            ffill[1 + slot] = t;
        }
    } else {
        if (n_empty > 0) {
            // step 6 at the few empty pixels.  E and K are only written here (at
            // empty pixels); the window maxima read C.
            const int Rl = p.large_radius;
            // their columns, in order (warps 0-2 take the bitmap's words)
            const unsigned w0 = ecols[0], w1 = ecols[1], w2 = ecols[2];
            if (tid < 96) {
                const int w = tid >> 5, lane = tid & 31;
                const unsigned bits = w == 0 ? w0 : (w == 1 ? w1 : w2);
                const int pos = (w > 0 ? __popc(w0) : 0) + (w > 1 ? __popc(w1) : 0) +
                                __popc(bits & ((1u << lane) - 1u));
                if ((bits >> lane) & 1u) {
                    ecol_list[pos] = tid;
                    ecol_idx[tid] = pos;
                }
            }
            const int ND = __popc(w0) + __popc(w1) + __popc(w2);
            const int lmin = w0 ? __ffs(w0) - 1 : (w1 ? 31 + __ffs(w1) : 63 + __ffs(w2));
            const int lmax = w2 ? 95 - __clz(w2) : (w1 ? 63 - __clz(w1) : 31 - __clz(w0));
            // the union of their windows: frame rows [by0, by1], columns [bx0, bx1]
            const int by0 = max(0, T.y0 - 4 + ebox[0] - Rl), by1 = min(H - 1, T.y0 - 4 + ebox[1] + Rl);
            const int bx0 = max(0, T.x0 - 4 + lmin - Rl), bx1 = min(W - 1, T.x0 - 4 + lmax + Rl);
            const int BR = by1 - by0 + 1, BC = bx1 - bx0 + 1;
            // row maxima at the ND empty columns (BR x ND), each column's top
            // and top value (2 x BC), then the box, which streams through the
            // rest of the scratch in bands of rows
            const int rm = BR * ND;
            const bool small = rm + 3 * BC <= kSmallScratch;
            const bool big = !small && rm + 3 * BC <= kBigScratch;
            if (small || big) {
                float* rmax = small ? scratch : reinterpret_cast<float*>(K);
                int* btop = reinterpret_cast<int*>(rmax + rm);
                float* btv = reinterpret_cast<float*>(btop + BC);
                float* band = btv + BC;
                const int RB = min(BR, ((small ? kSmallScratch : kBigScratch) - rm - 2 * BC) / BC);
                for (int c = tid; c < BC; c += kThreadsB) {
                    const int x = bx0 + c;
                    int top = kNoTop;
                    float tv = 0.0f;
                    if (p.extend_top) {
                        const unsigned long long t2 = __ldg(T.fd.top + x);
                        if (t2 != kNoTopPacked) {
                            top = (int)(t2 >> 32);
                            tv = top_value(T.fd, top, (unsigned)t2, x);
                        }
                    }
                    btop[c] = top;
                    btv[c] = tv;
                }
                __syncthreads();
                for (int r0 = 0; r0 < BR; r0 += RB) {
                    const int nb = min(RB, BR - r0);
                    // the band of E (step 5 applied): inside the tile's region from
                    // shared memory, elsewhere from C ...
                    for (int i = tid; i < nb * BC; i += kThreadsB) {
                        const int r = i / BC, c = i - r * BC;
                        const int k = by0 + r0 + r - (T.y0 - 4), l = bx0 + c - (T.x0 - 4);
                        band[i] = ((unsigned)k < (unsigned)kER && (unsigned)l < (unsigned)kEC)
                                      ? E[k * kES + l]
                                      : extended(T, p, by0 + r0 + r, bx0 + c, btop[c], btv[c]);
                    }
                    __syncthreads();
                    // ... its row maxima over the window width at the empty columns
                    for (int i = tid; i < nb * ND; i += kThreadsB) {
                        const int r = i / ND, j = i - r * ND;
                        const int c = T.x0 - 4 + ecol_list[j];
                        const int lo = max(c - Rl, bx0) - bx0, hi = min(c + Rl, bx1) - bx0;
                        float m = ninf();
                        for (int x = lo; x <= hi; ++x) m = fmaxf(m, band[r * BC + x]);
                        rmax[(r0 + r) * ND + j] = m;
                    }
                    __syncthreads();
                }
                // column maxima at each empty pixel
                for (int j = tid; j < n_empty; j += kThreadsB) {
                    const int k = elist[j] >> 16, l = elist[j] & 0xFFFF;
                    const int y = T.y0 - 4 + k;
                    const int lo = max(y - Rl, by0) - by0, hi = min(y + Rl, by1) - by0;
                    const int jc = ecol_idx[l];
                    float m = ninf();
                    for (int r = lo; r <= hi; ++r) m = fmaxf(m, rmax[r * ND + jc]);
                    E[k * kES + l] = m;
                    if (small) put_key(K, k, l, key_of(m, keys_ok));
                }
                if (big) {  // K held the row maxima: the keys again, from E
                    __syncthreads();
                    keys_ok = true;
                    build_keys(T, E, K, keys_ok);
                }
            } else {
                // too wide for the box: one warp per pixel, windows read from C
                const int warp = tid >> 5, lane = tid & 31;
                for (int j = warp; j < n_empty; j += kThreadsB / 32) {
                    const int k = elist[j] >> 16, l = elist[j] & 0xFFFF;
                    const float m = large_fill_at(T, p, T.y0 - 4 + k, T.x0 - 4 + l, lane);
                    if (lane == 0) {
                        E[k * kES + l] = m;
                        put_key(K, k, l, key_of(m, keys_ok));
                    }
                }
            }
            __syncthreads();
        }
        // replicate the frame border into the two rows / columns beyond each
        // edge (the median's rule; farther ones feed only mirrored outputs)
        if (T.y0 < 2 || T.x0 < 2 || T.y0 + kTBH + 2 > H || T.x0 + kTBW + 2 > W) {
            const Ring ring = ring_of(T, 4, kER, kEC);
            for (int i = tid; i < ring.count(); i += kThreadsB) {
                int k, l;
                ring.at(i, k, l);
                const int y = T.y0 - 4 + k, x = T.x0 - 4 + l;
                if (y < -2 || y >= H + 2 || x < -2 || x >= W + 2) continue;
                const int sk = clampi(y, H) - (T.y0 - 4), sl = clampi(x, W) - (T.x0 - 4);
                const float v = E[sk * kES + sl];
                E[k * kES + l] = v;
                put_key(K, k, l, key_of(v, keys_ok));
            }
        }
        const bool keys = __syncthreads_and(keys_ok);
        if (p.stop == kStopFillLarge) store_tile(E);
        else median_blur_store(T, p, E, K, keys, Mf, Mk, E);
    }
}

// Phase 1, persistent: CTA i starts with tile i and then takes the next
// unclaimed tile from a counter.  One region buffer and 16-bit median output
// (45 KB of shared memory in all) let five CTAs share an SM: while one waits
// for its region the others compute, which hides the copy better than a
// second buffer would (that costs CTAs per SM).  A tile runs on keys (C's
// key box, half the bytes of floats, moved into the median's packed layout
// by byte permutes) unless a value it needs is off the key grid, then on
// floats.  kFill: step 6 on (one instantiation per setting, so that neither
// carries the other's code: the kernel's speed is sensitive to its
// instruction footprint).  kInline: the step-6 worklist's tiles are done by
// the tile's CTA at once (for the capped or absent extension, where many
// tiles have many empty pixels; a kernel of its own otherwise: that code in
// this one slows the common case).
template <bool kFill, bool kInline>
__global__ void __launch_bounds__(kThreadsB, 5)
stage_b_main(const FrameDesc* __restrict__ frames, int n_frames, int total_tiles, StageBParams p,
             int* __restrict__ worklist, int* __restrict__ ffill, const __grid_constant__ CUtensorMap cmap,
             int* __restrict__ err)
{
    wait_previous_kernel();  // C, the tops and counters of stage A
    allow_next_kernel();
    extern __shared__ __align__(128) float smem[];  // the tensor copy wants 128-byte alignment
    __shared__ int ebox[2];
    MainSmem S;
    S.E = smem;
    S.K = reinterpret_cast<unsigned*>(smem + kER * kES);
    S.Mk = reinterpret_cast<unsigned short*>(S.K + kPR * kES);
    S.Mf = reinterpret_cast<float*>(S.K);
    S.scratch = reinterpret_cast<float*>(S.Mk);
    S.ctop = reinterpret_cast<int*>(S.scratch + kSmallScratch);
    S.ctv = reinterpret_cast<unsigned*>(S.ctop + kEC);
    S.elist = reinterpret_cast<int*>(S.ctv + kEC);
    S.ecount = S.elist + kMaxSparseFill;
    S.ecols = reinterpret_cast<unsigned*>(S.ecount + 4);
    S.ecol_list = reinterpret_cast<int*>(S.ecols + 4);
    S.ecol_idx = S.ecol_list + kEC;
    S.ebox = ebox;

    const int tid = threadIdx.x;
    int t = blockIdx.x;
    if (t >= total_tiles) return;
    Tile T = tile_of(frames, n_frames, t, p.row_stride);
    __shared__ int s_next;
    __shared__ __align__(8) unsigned long long s_mbar;  // completion of the region's tensor copy
    unsigned mbar_parity = 0;
    // the two block-wide tests of tile k, as bits of s_flags[k & 1]: 1 a
    // column top below the region's first row, 2 one at or above its last
    __shared__ unsigned s_flags[2];
    int k = 0;
    if (p.tma && tid == 0) mbar_init(&s_mbar);
    if (tid == 0) s_flags[0] = s_flags[1] = 0u;
    __syncthreads();
    for (;;) {
        const int H = T.fd.H, W = T.fd.W;
        if (p.tma) {
            if (tid == 0) tma_region(S.E, &cmap, key_box_x(T.x0), T.y0 - 4, T.f, &s_mbar);
        } else {
            issue_region_keys(T, reinterpret_cast<unsigned short*>(S.E));
        }
        load_tops(T, p, T.x0 - 4, kEC, S.ctop, S.ctv);
        reset_empties(S);
        if (tid == 0) s_next = (int)gridDim.x + atomicAdd(worklist + 1, 1);
        {
            // thread tid < kEC has just written column tid's top: its votes go
            // into the flag word now, and the region's barrier below publishes
            // them (the other word, tile k - 1's, was last read before this
            // tile began: cleared for tile k + 1)
            const int top = tid < kEC ? S.ctop[tid] : kNoTop;
            const bool below = tid < kEC && top != kNoTop && top > T.y0 - 4;
            const bool above = tid < kEC && (top == kNoTop || top <= T.y0 - 4 + kER - 1);
            const unsigned vb = __ballot_sync(0xffffffffu, below), va = __ballot_sync(0xffffffffu, above);
            if ((tid & 31) == 0 && (vb | va)) atomicOr(&s_flags[k & 1], (vb ? 1u : 0u) | (va ? 2u : 0u));
            if (tid == 0) s_flags[(k + 1) & 1] = 0u;
        }
        if (p.tma) {
            const bool arrived = mbar_wait(&s_mbar, mbar_parity);
            mbar_parity ^= 1u;
            if (!__syncthreads_and(arrived)) {  // the copy never completed: report, stop
                if (tid == 0) atomicOr(err, 1);
                return;
            }
        } else {
            cp_async_wait_all();
            __syncthreads();
        }
        const unsigned flags = s_flags[k & 1];
        ++k;
        // some column's top lies below the region's first row: step 5 writes
        const bool ext_tile = (flags & 1u) != 0u;
        const int tn = s_next;
        const bool more = tn < total_tiles;

        // a region entirely above its columns' tops: one row does for all
        const bool const_tile = p.extend_top && p.extend_rows < 0 && (flags & 2u) == 0u;
        // without step 6, a region empty in every column down to its last row
        // has an empty median everywhere (every window holds only empty
        // values): the tile's output is 0
        const bool void_tile = !kFill && p.stop == kStopFull &&
                               __syncthreads_and(tid >= kEC || column_empty_to(T, p, clampi(T.x0 - 4 + tid, W),
                                                                               min(H - 1, T.y0 - 4 + kER - 1)));
        if (const_tile) {
            tops_to_floats(T, T.x0 - 4, kEC, S.ctop, S.ctv);
            __syncthreads();
            constant_tile_store(T, p, reinterpret_cast<const float*>(S.ctv), S.scratch);
        } else if (void_tile) {
            store_zero_tile(T);
        } else if (!tile_keys<kFill, kInline>(T, p, S, t, worklist, ffill, ext_tile)) {
            tile_floats<kFill>(T, p, S, t, ffill, ext_tile);
        }

        __syncthreads();
        if (!more) break;
        T = tile_of(frames, n_frames, tn, p.row_stride);
        t = tn;
    }
}

// Row stride of the wide region in phase 2: 16-byte rows with room for the
// shift of the region's first column down to a 16-byte boundary.
__host__ __device__ constexpr int fill_row_stride(int GC) { return (GC + 6) / 4 * 4; }

// Row stride (in keys) of the wide key region of phase 2: the region's first
// column rounded down to a multiple of 8 (16-byte chunks) leaves up to 7
// keys before it; a multiple of 8.
__host__ __device__ constexpr int fill_key_stride(int GC) { return (GC + 14) / 8 * 8; }

// Bytes of the wide key region, also the Gaussian's row-pass buffer later.
__host__ __device__ constexpr size_t fill_key_gbytes(int large_radius)
{
    const size_t g = (size_t)(kER + 2 * large_radius) * fill_key_stride(kEC + 2 * large_radius) * 2;
    const size_t r = (size_t)kMR * kRS * sizeof(float);
    return ((g > r ? g : r) + 15) / 16 * 16;
}

// Step 6 and the rest of the chain for tile t (T) of the step-6 worklist,
// in shared memory from dynk (stage_b_fill_keys_smem_bytes of it; the
// caller's block has synchronised, and any earlier use of it is over).
__device__ void fill_tile_keys(const Tile& T, int t, const StageBParams& p, unsigned char* __restrict__ dynk,
                               int* __restrict__ ffill)
{
    const int Rl = p.large_radius;
    const int GR = kER + 2 * Rl, GC = kEC + 2 * Rl;
    const int GSk = fill_key_stride(GC), GSW = GSk / 2;  // keys, words per row
    unsigned short* Gk = reinterpret_cast<unsigned short*>(dynk);
    unsigned* Gw = reinterpret_cast<unsigned*>(dynk);
    float* R = reinterpret_cast<float*>(dynk);
    unsigned* K = reinterpret_cast<unsigned*>(dynk + fill_key_gbytes(Rl));
    unsigned short* Mk = reinterpret_cast<unsigned short*>(K + kPR * kES);
    int* ctop = reinterpret_cast<int*>(Mk + kMR * kMS);
    unsigned* ctv = reinterpret_cast<unsigned*>(ctop + GC);
    const int tid = threadIdx.x;
    const int wl = 2 * Rl + 1;
    const int H = T.fd.H, W = T.fd.W;
    const int gy = T.y0 - 4 - Rl, gx = T.x0 - 4 - Rl;  // frame position of the wide region's (0, 0)
    const int gxa = gx & ~7, sh = gx - gxa;            // buffer column b is frame column gxa + b
    load_tops(T, p, gx, GC, ctop, ctv);
    // a wide region empty in every column: every window of step 6 holds
    // only empty values, so does the median, and the output is 0
    if (p.stop == kStopFull) {
        bool empty_cols = true;
        const int last = min(H - 1, gy + GR - 1);
        for (int l = tid; l < GC; l += kThreadsB) {
            const int x = gx + l;
            if (x >= 0 && x < W) empty_cols = empty_cols && column_empty_to(T, p, x, last);
        }
        if (__syncthreads_and(empty_cols)) {
            store_zero_tile(T);
            return;
        }
    }
    // C's keys over the wide region's rows, whole 16-byte chunks inside the
    // frame, the rest key by key with 0 outside the frame
    const int nch = GSk / 8;
    for (int i = tid; i < GR * nch; i += kThreadsB) {
        const int k = i / nch, j = i - k * nch;
        const int y = gy + k, x = gxa + 8 * j;
        unsigned short* dst = Gk + k * GSk + 8 * j;
        if (y >= 0 && y < H && x >= 0 && x + 8 <= W) {
            cp_async16(dst, T.fd.ck + (size_t)y * T.fd.c_pitch + x);
        } else {
            const bool row_in = y >= 0 && y < H;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                dst[e] = (row_in && x + e >= 0 && x + e < W) ? T.fd.ck[(size_t)y * T.fd.c_pitch + x + e]
                                                             : (unsigned short)0;
        }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    // step 5: the rows above each in-frame column's top (within the cap)
    if (p.extend_top) {
        for (int l = tid; l < GC; l += kThreadsB) {
            const int top = ctop[l], x = gx + l;
            if (top == kNoTop || x < 0 || x >= W) continue;
            const int klo = max(-gy, p.extend_rows < 0 ? 0 : top - p.extend_rows - gy);
            const int khi = min(GR, top - gy);
            const unsigned short v = (unsigned short)ctv[l];
            for (int k = max(0, klo); k < khi; ++k) Gk[k * GSk + sh + l] = v;
        }
        __syncthreads();
    }
    // a value off the key grid anywhere in the buffer: the float pass does the tile
    unsigned mx = 0u;
    for (int i = tid; i < GR * GSW; i += kThreadsB) mx = __vmaxu2(mx, Gw[i]);
    if (__syncthreads_or((mx & 0xFFFFu) > kKeyMax || (mx >> 16) > kKeyMax)) {
        if (tid == 0) {
            const int slot = atomicAdd(ffill, 1);
            ffill[1 + slot] = t;
        }
        return;
    }
    // K: E over tile + 4, border replicated, rows (kp, kp + kHalf) per word;
    // thread t < kRowGroups x kChunksPerRow takes column chunk t %
    // kChunksPerRow of every kRowGroups-th K row
    const int g = tid / kChunksPerRow, q = tid - g * kChunksPerRow;
    if (tid < kRowGroups * kChunksPerRow) {
        int bcol[4];  // buffer columns of the chunk (clamped into the frame)
#pragma unroll
        for (int e = 0; e < 4; ++e) bcol[e] = clampi(T.x0 - 4 + 4 * q + e, W) - gxa;
        for (int kp = g; kp < kPR; kp += kRowGroups) {
            const unsigned short* ra = Gk + (clampi(T.y0 - 4 + kp, H) - gy) * GSk;
            const unsigned short* rb = Gk + (clampi(T.y0 - 4 + kp + kHalf, H) - gy) * GSk;
            unsigned wd[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) wd[e] = (unsigned)ra[bcol[e]] | ((unsigned)rb[bcol[e]] << 16);
            *reinterpret_cast<uint4*>(K + kp * kES + 4 * q) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
    }
    __syncthreads();
    // window maxima down the columns, in place (van Herk / Gil-Werman):
    // rows [0, kER) end with the maximum over [r, r + 2 Rl].  In blocks of
    // wl rows: going down block [b0, b0 + wl) from its end, each row takes
    // the maximum from it to the block's end; going up again, row b0 + i
    // takes the larger of that and the maximum of the next block's first i
    // rows, which is its window.  The next block is overwritten only after
    // this one is done.  One thread per word column (two columns each).
    {
        const int wc0 = sh >> 1, wc1 = (sh + GC + 1) >> 1;
        for (int wc = wc0 + tid; wc < wc1; wc += kThreadsB) {
            unsigned* col = Gw + wc;
            for (int b0 = 0; b0 < kER; b0 += wl) {
                unsigned h = 0u;
#pragma unroll 4
                for (int r = b0 + wl - 1; r >= b0; --r) {
                    h = __vmaxu2(h, col[r * GSW]);
                    col[r * GSW] = h;
                }
                const int n = min(wl, kER - b0);
                unsigned g = 0u;
                col[b0 * GSW] = h;  // i = 0: the block itself
#pragma unroll 4
                for (int i = 1; i < n; ++i) {
                    g = __vmaxu2(g, col[(b0 + wl + i - 1) * GSW]);
                    col[(b0 + i) * GSW] = __vmaxu2(col[(b0 + i) * GSW], g);
                }
            }
        }
    }
    __syncthreads();
    // window maxima along the rows [0, kER), in place by the same scheme:
    // region columns [0, kEC) end with the maximum over [l, l + 2 Rl].  One
    // thread per row; a row's blocks start at column o (0..14 by the
    // thread's lane, so that at each step the rows of a warp reach
    // different banks: at the paper's 31 x 31 the rows are 24 words mod 32
    // apart), and columns [0, o) are a head block before them.
    if (tid < kER) {
        unsigned short* x = Gk + tid * GSk + sh;
        const int o = min(2 * ((tid & 31) >> 2), wl - 1);
        if (o > 0) {
            unsigned h = 0u;
            for (int l = o - 1; l >= 0; --l) {
                h = max(h, (unsigned)x[l]);
                x[l] = (unsigned short)h;
            }
            unsigned g = 0u;  // block 0's columns before the first window's end
            for (int l = o; l < wl - 1; ++l) g = max(g, (unsigned)x[l]);
            for (int l = 0; l < o; ++l) {
                g = max(g, (unsigned)x[l + wl - 1]);
                x[l] = (unsigned short)max((unsigned)x[l], g);
            }
        }
        for (int b0 = o; b0 < kEC; b0 += wl) {
            unsigned h = 0u;
#pragma unroll 4
            for (int l = b0 + wl - 1; l >= b0; --l) {
                h = max(h, (unsigned)x[l]);
                x[l] = (unsigned short)h;
            }
            const int n = min(wl, kEC - b0);
            unsigned g = 0u;
#pragma unroll 4
            for (int i = 1; i < n; ++i) {
                g = max(g, (unsigned)x[b0 + wl + i - 1]);
                x[b0 + i] = (unsigned short)max((unsigned)x[b0 + i], g);
            }
        }
    }
    __syncthreads();
    // step 6: an empty position takes the maximum at its window's corner
    // (the clamped pixel's, at the replicated border)
    if (tid < kRowGroups * kChunksPerRow) {
        // a window's corner column is the clamped column - Rl, in buffer columns
        int bcol[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) bcol[e] = clampi(T.x0 - 4 + 4 * q + e, W) - gxa - Rl;
        for (int kp = g; kp < kPR; kp += kRowGroups) {
            uint4* cell = reinterpret_cast<uint4*>(K + kp * kES + 4 * q);
            uint4 c4 = *cell;
            unsigned wd[4] = {c4.x, c4.y, c4.z, c4.w};
            const unsigned mn = __vminu2(__vimin3_u16x2(wd[0], wd[1], wd[2]), wd[3]);
            if ((mn & 0xFFFFu) > kEmptyKeyMax && (mn >> 16) > kEmptyKeyMax) continue;  // nothing empty
            const unsigned short* ga = Gk + (clampi(T.y0 - 4 + kp, H) - gy - Rl) * GSk;
            const unsigned short* gb = Gk + (clampi(T.y0 - 4 + kp + kHalf, H) - gy - Rl) * GSk;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if ((wd[e] & 0xFFFFu) <= kEmptyKeyMax) wd[e] = (wd[e] & 0xFFFF0000u) | ga[bcol[e]];
                if ((wd[e] >> 16) <= kEmptyKeyMax) wd[e] = (wd[e] & 0xFFFFu) | ((unsigned)gb[bcol[e]] << 16);
            }
            *cell = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
    }
    __syncthreads();
    if (p.stop == kStopFillLarge) {
        store_keys_tile(T, K);
        return;
    }
    median_blur_store(T, p, nullptr, K, true, reinterpret_cast<float*>(K), Mk, R);
}

// Phase 2 on keys: the tiles with more empty pixels than a tile fills
// itself (worklist[0] of them from worklist[3]), with step 6.  The wide
// region (tile + 4 + the window radius) of C's keys arrives by 16-byte
// cp.async chunks (the few across the frame's edges by plain loads, key 0
// outside it), step 5 is applied per column, and K (the median's packed
// layout) takes E over tile + 4, border replicated.  The window maxima are
// taken in place by van Herk and Gil-Werman's scheme (three maxima per
// value whatever the window: per block of wl values the maxima to the
// block's end, then those combined with the running maxima of the next
// block's start): down the columns on packed words (two columns each), one
// thread per word column, then along the rows on keys, one thread per row.
// K's empty positions take the maximum at their window's corner;
// then the packed median, the exact blur on keys and the store.  A tile
// whose region holds a value off the key grid goes to the float list
// (ffill[0] of them from ffill[1]) for stage_b_fill.  About 41 KB of shared
// memory at the paper's 31 x 31: five CTAs per SM.
__global__ void __launch_bounds__(kThreadsB, 5)
stage_b_fill_keys(const FrameDesc* __restrict__ frames, int n_frames, StageBParams p,
                  const int* __restrict__ worklist, int* __restrict__ ffill)
{
    wait_previous_kernel();  // the worklist and outputs of the main pass
    allow_next_kernel();
    extern __shared__ __align__(16) unsigned char dynk[];
    const int count = worklist[0];
    for (int w = blockIdx.x; w < count; w += gridDim.x) {
        __syncthreads();
        const int t = worklist[3 + w];
        fill_tile_keys(tile_of(frames, n_frames, t, p.row_stride), t, p, dynk, ffill);
    }
}

// Phase 2 on floats: the tiles with many empty pixels whose values are off
// the key grid, from the float list (ffill[0] of them from ffill[1]), with
// step 6.  Shared memory: G (E over
// the wide region, rows of GS floats, 16-byte aligned, frame column gx at
// offset sh; the window maxima are taken in place there, then it holds the
// median output), F (E, then the step-6 output, over tile + 4; the blur's
// buffer once the median has read it) and the region's column tops.  About
// 60 KB at the paper's 31 x 31: three CTAs per SM.
__global__ void __launch_bounds__(kThreadsB, 3)
stage_b_fill(const FrameDesc* __restrict__ frames, int n_frames, StageBParams p,
             const int* __restrict__ ffill)
{
    wait_previous_kernel();  // the list and outputs of the main pass and of the key pass
    extern __shared__ __align__(16) float dyn[];
    const int Rl = p.large_radius;
    const int GR = kER + 2 * Rl, GC = kEC + 2 * Rl;  // the wide region
    const int GS = fill_row_stride(GC);
    float* G = dyn;
    float* F = G + GR * GS;
    float* M = G;
    int* ctop = reinterpret_cast<int*>(F + kER * kES);
    unsigned* ctv = reinterpret_cast<unsigned*>(ctop + GC);
    const float* cval = reinterpret_cast<const float*>(ctv);  // after tops_to_floats
    float* R = F;

    const int count = ffill[0];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int w = blockIdx.x; w < count; w += gridDim.x) {
        __syncthreads();
        const Tile T = tile_of(frames, n_frames, ffill[1 + w], p.row_stride);
        const int H = T.fd.H, W = T.fd.W;
        const int gy = T.y0 - 4 - Rl, gx = T.x0 - 4 - Rl;  // frame position of the wide region's (0, 0)
        load_tops(T, p, gx, GC, ctop, ctv);
        // a wide region empty in every column: every window of step 6 holds
        // only empty values, so does the median, and the output is 0
        if (p.stop == kStopFull) {
            bool empty_cols = true;
            const int last = min(H - 1, gy + GR - 1);
            for (int l = tid; l < GC; l += kThreadsB) {
                const int x = gx + l;
                if (x >= 0 && x < W) empty_cols = empty_cols && column_empty_to(T, p, x, last);
            }
            if (__syncthreads_and(empty_cols)) {
                store_zero_tile(T);
                continue;
            }
        }
        tops_to_floats(T, gx, GC, ctop, ctv);
        // E over the wide region: C from its keys (and the float map), -inf
        // outside the frame
        constexpr int sh = 0;  // frame column gx at row offset 0
        for (int k = warp; k < GR; k += kThreadsB / 32) {
            const int y = gy + k;
            float* grow = G + k * GS;
            if (y < 0 || y >= H) {
                for (int j = lane; j < GS; j += 32) grow[j] = ninf();
                continue;
            }
            for (int j = lane; j < GC; j += 32) {
                const int x = gx + j;
                grow[j] = (x >= 0 && x < W) ? c_at(T.fd, y, x) : ninf();
            }
        }
        __syncthreads();
        // step 5: the rows above each in-frame column's top (within the cap)
        if (p.extend_top) {
            for (int l = tid; l < GC; l += kThreadsB) {
                const int top = ctop[l], x = gx + l;
                if (top == kNoTop || x < 0 || x >= W) continue;
                const int klo = max(-gy, p.extend_rows < 0 ? 0 : top - p.extend_rows - gy);
                const int khi = min(GR, top - gy);
                const float v = cval[l];
                for (int k = max(0, klo); k < khi; ++k) G[k * GS + sh + l] = v;
            }
            __syncthreads();
        }
        // E over tile + 4, border replicated, kept in F: G is scratch below
        for (int i = tid; i < kER * kEC; i += kThreadsB) {
            const int k = i / kEC, l = i - k * kEC;
            const int y = clampi(T.y0 - 4 + k, H), x = clampi(T.x0 - 4 + l, W);
            F[k * kES + l] = G[(y - gy) * GS + sh + (x - gx)];
        }
        // The window maxima, separable and in place, by van Herk and
        // Gil-Werman's scheme (as on keys in stage_b_fill_keys): G is E over
        // the wide region; F keeps E over tile + 4 for the fill below.
        __syncthreads();
        const int wl = 2 * Rl + 1;
        // columns, one thread each (neighbouring threads, neighbouring banks):
        // rows [0, kER) end with the maximum over [r, r + 2 Rl]
        for (int c = tid; c < GC; c += kThreadsB) {
            float* __restrict__ col = G + sh + c;
            for (int b0 = 0; b0 < kER; b0 += wl) {
                float h = ninf();
#pragma unroll 4
                for (int r = b0 + wl - 1; r >= b0; --r) {
                    h = fmaxf(h, col[r * GS]);
                    col[r * GS] = h;
                }
                const int n = min(wl, kER - b0);
                float g = ninf();
#pragma unroll 4
                for (int i = 1; i < n; ++i) {
                    g = fmaxf(g, col[(b0 + wl + i - 1) * GS]);
                    col[(b0 + i) * GS] = fmaxf(col[(b0 + i) * GS], g);
                }
            }
        }
        __syncthreads();
        // rows [0, kER), one thread each, columns [0, kEC) end with the maximum
        // over [c, c + 2 Rl]; a row's blocks start at column o (0..7 by the
        // thread's lane: at the paper's 31 x 31 the rows are 8 banks apart),
        // columns [0, o) a head block before them
        if (tid < kER) {
            float* __restrict__ x = G + tid * GS + sh;
            const int o = min((tid & 31) >> 2, wl - 1);
            if (o > 0) {
                float h = ninf();
                for (int l = o - 1; l >= 0; --l) {
                    h = fmaxf(h, x[l]);
                    x[l] = h;
                }
                float g = ninf();  // block 0's columns before the first window's end
                for (int l = o; l < wl - 1; ++l) g = fmaxf(g, x[l]);
                for (int l = 0; l < o; ++l) {
                    g = fmaxf(g, x[l + wl - 1]);
                    x[l] = fmaxf(x[l], g);
                }
            }
            for (int b0 = o; b0 < kEC; b0 += wl) {
                float h = ninf();
#pragma unroll 4
                for (int l = b0 + wl - 1; l >= b0; --l) {
                    h = fmaxf(h, x[l]);
                    x[l] = h;
                }
                const int n = min(wl, kEC - b0);
                float g = ninf();
#pragma unroll 4
                for (int i = 1; i < n; ++i) {
                    g = fmaxf(g, x[b0 + wl + i - 1]);
                    x[b0 + i] = fmaxf(x[b0 + i], g);
                }
            }
        }
        __syncthreads();
        // the fill of empty pixels, tile + 4, replicated border
        for (int i = tid; i < kER * kEC; i += kThreadsB) {
            const int k = i / kEC, l = i - k * kEC;
            const int y = clampi(T.y0 - 4 + k, H), x = clampi(T.x0 - 4 + l, W);
            const int dk = y - gy - Rl, dl = x - gx - Rl;  // the window's corner
            const float e = F[k * kES + l];
            if (is_empty(e)) F[k * kES + l] = fmaxf(e, G[dk * GS + sh + dl]);
        }
        __syncthreads();
        if (p.stop == kStopFillLarge) {
            for (int i = tid; i < kTBH * kTBW; i += kThreadsB) {
                const int a = i / kTBW, b = i - a * kTBW;
                const int y = T.y0 + a, x = T.x0 + b;
                if (y < H && x < W) T.fd.out[(size_t)y * T.fd.out_pitch + x] = F[(a + 4) * kES + b + 4];
            }
            continue;
        }
        median_blur_store(T, p, F, nullptr, false, M, nullptr, R);
    }
}

}  // namespace

size_t stage_b_fill_smem_bytes(int large_radius)
{
    const int GR = kER + 2 * large_radius, GC = kEC + 2 * large_radius;
    return sizeof(float) * ((size_t)GR * fill_row_stride(GC) + kER * kES + 2 * GC);
}

size_t stage_b_fill_keys_smem_bytes(int large_radius)
{
    return fill_key_gbytes(large_radius) + sizeof(unsigned) * kPR * kES + sizeof(unsigned short) * kMR * kMS +
           2 * sizeof(int) * (kEC + 2 * large_radius);
}

// As many CTAs per SM of a kernel as shared memory and registers hold.
template <class Kern>
int occupancy_ctas(Kern kernel, size_t smem)
{
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreadsB, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n < 1 ? 1 : n;
}

cudaError_t preload_stage_b()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, stage_b_main<true, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_b_main<true, true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_b_main<false, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_b_fill_keys);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_b_fill);
    return e;
}

namespace {
// The main pass does the step-6 worklist's tiles itself when the extension
// is capped or off (then many tiles have many empty pixels) and their wide
// region fits in its shared memory (windows up to 43 x 43, the paper's 31 x
// 31 among them): that saves the worklist kernel's launch and spreads the
// worklist's tiles over the main pass.  Otherwise stage_b_fill_keys.
bool fill_inline(const StageBParams& p)
{
    return p.large_fill_on && (!p.extend_top || p.extend_rows >= 0) &&
           stage_b_fill_keys_smem_bytes(p.large_radius) <= sizeof(float) * kMainSmemFloats;
}
}  // namespace

int stage_b_launches(const StageBParams& p)
{
    if (!p.large_fill_on || p.stop == kStopExtend) return 1;
    return fill_inline(p) ? 2 : 3;
}

cudaError_t launch_stage_b(const FrameDesc* d_frames, int n_frames, int total_tiles,
                           const StageBParams& p, int* worklist, int* ffill, int sm_count, int ctas_per_sm,
                           const CUtensorMap* cmap, int* err, cudaStream_t stream)
{
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t main_smem = sizeof(float) * kMainSmemFloats;
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(stage_b_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)stage_b_fill_smem_bytes(kMaxLargeFill / 2));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(stage_b_fill_keys, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)stage_b_fill_keys_smem_bytes(kMaxLargeFill / 2));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(stage_b_main<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)main_smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(stage_b_main<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)main_smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(stage_b_main<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)main_smem);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    if (total_tiles < 1) return cudaSuccess;
    if (ctas_per_sm < 1) ctas_per_sm = 1;
    if (ctas_per_sm > 5) ctas_per_sm = 5;  // shared memory and registers hold five per SM
    const int main_grid = total_tiles < ctas_per_sm * sm_count ? total_tiles : ctas_per_sm * sm_count;
    CUtensorMap map{};
    if (p.tma && cmap) map = *cmap;
    StageBParams q = p;
    q.tma = (p.tma && cmap) ? 1 : 0;
    q.fill_inline = fill_inline(p) ? 1 : 0;
    cudaError_t e = launch_after_previous(!p.large_fill_on ? stage_b_main<false, false>
                                          : q.fill_inline  ? stage_b_main<true, true>
                                                           : stage_b_main<true, false>,
                                          dim3(main_grid), dim3(kThreadsB), main_smem, stream, d_frames, n_frames,
                                          total_tiles, q, worklist, ffill, map, err);
    if (e != cudaSuccess || !p.large_fill_on || p.stop == kStopExtend) return e;
    // step 6 over the worklist on keys (unless the main pass did its tiles),
    // then on floats over the tiles off the key grid
    int grid = 0;
    if (!q.fill_inline) {
        const size_t kfill_smem = stage_b_fill_keys_smem_bytes(p.large_radius);
        grid = occupancy_ctas(stage_b_fill_keys, kfill_smem) * sm_count;
        if (grid > total_tiles) grid = total_tiles;
        e = launch_after_previous(stage_b_fill_keys, dim3(grid), dim3(kThreadsB), kfill_smem, stream, d_frames,
                                  n_frames, q, static_cast<const int*>(worklist), ffill);
        if (e != cudaSuccess) return e;
    }
    const size_t fill_smem = stage_b_fill_smem_bytes(p.large_radius);
    grid = occupancy_ctas(stage_b_fill, fill_smem) * sm_count;
    if (grid > total_tiles) grid = total_tiles;
    return launch_after_previous(stage_b_fill, dim3(grid), dim3(kThreadsB), fill_smem, stream, d_frames, n_frames, q,
                                 static_cast<const int*>(ffill));
}

}  // namespace dcgb
