// stage_a_float.cuh -- steps 1-4 of arXiv 1802.00036, Section IV, on floats,
// streamed down column strips: one unit (a strip over a band of rows) per
// warp.  Shared by the float kernel (stage_a.cu) and the key kernel
// (stage_a_keys.cu), which runs it on its units whose inputs are off the
// key grid.
//
// One warp owns a strip of 32 x kV adjacent columns (lane l holds columns
// kV*l .. kV*l + kV - 1) and walks down a band of rows, one input row per
// step.  Every vertical window lives in small register rings; the horizontal
// part of every window comes from the lane's own columns plus up to three
// columns of each neighbouring lane (warp shuffles).  The steps are
//   1  invert: 100 - d on valid pixels (one float32 subtraction), 0 else;
//   2  the first element (Fig. 4) as row maxima of half-width 0..3 combined
//      over its rows;
//   3  5x5 close: 5-wide row max, 5-row max, 5-wide row min, 5-row min;
//   4  7x7 max (7-wide, 7-row) written into empty pixels only;
// with 3-input min/max (one instruction on sm_103a).  Each step delays its
// output by its vertical radius, so step 4 emits row t - (r1 + 7) when input
// row t arrives.  A pixel outside the frame holds the neutral value of the
// operation that reads it (-inf before a max, +inf before a min), which is
// "out-of-frame pixels are ignored".  The strip's outer r1 + 7 columns on
// each side are only halo: strips overlap by that much, bands by as many
// rows, and the rings start with values that only reach rows above the band.
//
// Output: C (the step-4 map) into scratch as 16-bit keys (k for a value
// k / 256; a value off that grid as kKeyOff, the value itself in the float
// map), and for each column the smallest row with a non-empty C and its key,
// by a 64-bit atomicMin on top[] (step 5 needs them).  With a stop before
// step 5 the requested map goes to the output instead.
#pragma once

#include "common.cuh"

#include <climits>
#include <type_traits>

namespace dcgb {
namespace {
namespace afloat {

constexpr int kV = kStageAColsPerLane;
constexpr int kSW = 32 * kV;  // strip width in columns

__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// A row of kV values plus up to three neighbours on each side.
struct Row {
    float v[kV];
    float l[4];  // l[i]: column -i  (l[0] unused)
    float r[4];  // r[i]: column kV - 1 + i (r[0] unused)
    __device__ __forceinline__ float at(int j) const
    {
        return j < 0 ? l[-j] : (j >= kV ? r[j - kV + 1] : v[j]);
    }
};

// Fetch `rad` neighbour columns on each side from the adjacent lanes.  In a
// strip that starts at the frame's first column (at_left, warp-uniform) the
// columns left of lane 0 are outside the frame: the operation's neutral value.
template <int rad>
__device__ __forceinline__ void neighbours(Row& x, bool at_left, float neutral)
{
#pragma unroll
    for (int i = 1; i <= rad; ++i) {
        x.l[i] = __shfl_up_sync(0xffffffffu, x.v[kV - i], 1);
        x.r[i] = __shfl_down_sync(0xffffffffu, x.v[i - 1], 1);
    }
    if (at_left && (threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 1; i <= rad; ++i) x.l[i] = neutral;
}

template <bool kMax>
__device__ __forceinline__ float ext3(float a, float b, float c)
{
    return kMax ? max3f(a, b, c) : min3f(a, b, c);
}

template <int S> struct ShapeInfo;
template <> struct ShapeInfo<kDiamond5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kFull5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kCross5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kFull3> { static constexpr int r = 1; };
template <> struct ShapeInfo<kCircle5> { static constexpr int r = 2; };
template <> struct ShapeInfo<kFull7> { static constexpr int r = 3; };

// 7-row window of a row extreme h: u(o) = ext(h(o-2), h(o-1), h(o));
// out(o-3) = ext(u(o-4), u(o-1), h(o)).
template <bool kMax>
struct Window7 {
    float h[2][kV], u[4][kV];
    __device__ void init(float fill)
    {
        for (int v = 0; v < kV; ++v) {
            h[0][v] = h[1][v] = fill;
            u[0][v] = u[1][v] = u[2][v] = u[3][v] = fill;
        }
    }
    template <int PHI>
    __device__ __forceinline__ float push(int v, float hn)
    {
        const float un = ext3<kMax>(h[PHI & 1][v], h[(PHI + 1) & 1][v], hn);
        const float o = ext3<kMax>(u[PHI & 3][v], u[(PHI + 3) & 3][v], hn);
        h[PHI & 1][v] = hn;
        u[PHI & 3][v] = un;
        return o;
    }
};

// Step 2 for each element: rings of the rows it still needs; push() takes
// input row t and returns the dilation of row t - r1.
template <int S> struct FirstDilation;

template <> struct FirstDilation<kDiamond5> {
    // rows: |dy| = 2 -> width 1, |dy| = 1 -> 3, dy = 0 -> 5
    // p(o) = max(x(o-2), h1(o-1), h2(o));  A(o) = max(p(o), h1(o+1), x(o+2))
    float x[2][kV], p[2][kV], h1[kV];
    __device__ void init()
    {
        for (int v = 0; v < kV; ++v) x[0][v] = x[1][v] = p[0][v] = p[1][v] = h1[v] = ninf();
    }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<2>(in, at_left, ninf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float a1 = max3f(in.at(v - 1), in.v[v], in.at(v + 1));
            const float a2 = max3f(a1, in.at(v - 2), in.at(v + 2));
            const float pn = max3f(x[PHI & 1][v], h1[v], a2);
            out[v] = max3f(p[PHI & 1][v], h1[v], in.v[v]);
            x[PHI & 1][v] = in.v[v];
            p[PHI & 1][v] = pn;
            h1[v] = a1;
        }
    }
};

template <> struct FirstDilation<kFull5> {
    // 5-wide row max h; s(o) = max(h(o-2), h(o-1), h(o)); A(o-2) = max(s(o-2), h(o-1), h(o))
    float h[2][kV], s[2][kV];
    __device__ void init()
    {
        for (int v = 0; v < kV; ++v) h[0][v] = h[1][v] = s[0][v] = s[1][v] = ninf();
    }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<2>(in, at_left, ninf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float a2 = max3f(max3f(in.at(v - 2), in.at(v - 1), in.v[v]), in.at(v + 1), in.at(v + 2));
            const float hm1 = h[(PHI + 1) & 1][v], hm2 = h[PHI & 1][v];
            out[v] = max3f(s[PHI & 1][v], hm1, a2);
            s[PHI & 1][v] = max3f(hm2, hm1, a2);
            h[PHI & 1][v] = a2;
        }
    }
};

template <> struct FirstDilation<kCross5> {
    // p(o) = max(x(o-2), x(o-1), h2(o));  A(o) = max(p(o), x(o+1), x(o+2))
    float x[2][kV], p[2][kV];
    __device__ void init()
    {
        for (int v = 0; v < kV; ++v) x[0][v] = x[1][v] = p[0][v] = p[1][v] = ninf();
    }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<2>(in, at_left, ninf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float a2 = max3f(max3f(in.at(v - 2), in.at(v - 1), in.v[v]), in.at(v + 1), in.at(v + 2));
            const float xm1 = x[(PHI + 1) & 1][v], xm2 = x[PHI & 1][v];
            const float pn = max3f(xm2, xm1, a2);
            out[v] = max3f(p[PHI & 1][v], xm1, in.v[v]);
            x[PHI & 1][v] = in.v[v];
            p[PHI & 1][v] = pn;
        }
    }
};

template <> struct FirstDilation<kFull3> {
    // A(o-1) = max(h1(o-2), h1(o-1), h1(o))
    float h[2][kV];
    __device__ void init()
    {
        for (int v = 0; v < kV; ++v) h[0][v] = h[1][v] = ninf();
    }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<1>(in, at_left, ninf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float a1 = max3f(in.at(v - 1), in.v[v], in.at(v + 1));
            out[v] = max3f(h[PHI & 1][v], h[(PHI + 1) & 1][v], a1);
            h[PHI & 1][v] = a1;
        }
    }
};

template <> struct FirstDilation<kCircle5> {
    // rows: |dy| = 2 -> width 3, |dy| <= 1 -> 5
    // p(o) = max(h1(o-2), h2(o-1), h2(o));  A(o) = max(p(o), h2(o+1), h1(o+2))
    float h1[2][kV], h2[kV], p[2][kV];
    __device__ void init()
    {
        for (int v = 0; v < kV; ++v) h1[0][v] = h1[1][v] = h2[v] = p[0][v] = p[1][v] = ninf();
    }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<2>(in, at_left, ninf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float a1 = max3f(in.at(v - 1), in.v[v], in.at(v + 1));
            const float a2 = max3f(a1, in.at(v - 2), in.at(v + 2));
            const float pn = max3f(h1[PHI & 1][v], h2[v], a2);
            out[v] = max3f(p[PHI & 1][v], h2[v], a1);
            h1[PHI & 1][v] = a1;
            h2[v] = a2;
            p[PHI & 1][v] = pn;
        }
    }
};

template <> struct FirstDilation<kFull7> {
    Window7<true> w;
    __device__ void init() { w.init(ninf()); }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<3>(in, at_left, ninf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float a3 = max3f(max3f(in.at(v - 3), in.at(v - 2), in.at(v - 1)), in.v[v],
                                   max3f(in.at(v + 1), in.at(v + 2), in.at(v + 3)));
            out[v] = w.template push<PHI>(v, a3);
        }
    }
};

// 5x5 square max or min: 5-wide row extreme h, then
// s(o) = ext(h(o-2), h(o-1), h(o)); out(o-2) = ext(s(o-2), h(o-1), h(o)).
template <bool kMax>
struct Square5 {
    float h[2][kV], s[2][kV];
    __device__ void init(float fill)
    {
        for (int v = 0; v < kV; ++v) h[0][v] = h[1][v] = s[0][v] = s[1][v] = fill;
    }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<2>(in, at_left, kMax ? ninf() : pinf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float hn =
                ext3<kMax>(ext3<kMax>(in.at(v - 2), in.at(v - 1), in.v[v]), in.at(v + 1), in.at(v + 2));
            const float hm1 = h[(PHI + 1) & 1][v], hm2 = h[PHI & 1][v];
            out[v] = ext3<kMax>(s[PHI & 1][v], hm1, hn);
            s[PHI & 1][v] = ext3<kMax>(hm2, hm1, hn);
            h[PHI & 1][v] = hn;
        }
    }
};

// Step 4: 7x7 max written into empty pixels of B only.
struct Fill7 {
    Window7<true> w;
    float b[4][kV];  // B rows, to select C(o - 3)
    __device__ void init()
    {
        w.init(ninf());
        for (int v = 0; v < kV; ++v) b[0][v] = b[1][v] = b[2][v] = b[3][v] = ninf();
    }
    template <int PHI>
    __device__ __forceinline__ void push(Row& in, float (&out)[kV], bool at_left)
    {
        neighbours<3>(in, at_left, ninf());
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float hn = max3f(max3f(in.at(v - 3), in.at(v - 2), in.at(v - 1)), in.v[v],
                                   max3f(in.at(v + 1), in.at(v + 2), in.at(v + 3)));
            const float m7 = w.template push<PHI>(v, hn);
            const float bc = b[(PHI + 1) & 3][v];  // B(o - 3)
            out[v] = is_empty(bc) ? m7 : bc;
            b[PHI & 3][v] = in.v[v];
        }
    }
};

// One unit (a strip of kSW columns over one band of rows) of steps 1-4.
template <int S>
__device__ __forceinline__ void stage_a_unit(const FrameDesc* __restrict__ frames, int n_frames, int unit,
                                             int stop, int band_stride)
{
    constexpr int R1 = ShapeInfo<S>::r;
    constexpr int Rh = R1 + 7;        // halo, horizontal and vertical
    const int lane = threadIdx.x & 31;
    // Bands from the bottom up (the rows with data, the costly ones, come
    // first): with frames of one shape (band_stride = strips of the batch)
    // the batch's bottom bands, then the next ones up; else frame by frame.
    int f, band, strip;
    if (band_stride > 0) {
        const int r = unit / band_stride, g = unit - r * band_stride;
        f = g / frames[0].tiles_x_a;
        strip = g - f * frames[0].tiles_x_a;
        band = (frames[0].H + frames[0].band_a - 1) / frames[0].band_a - 1 - r;
    } else {
        f = find_frame<true>(frames, n_frames, unit);
        const int local = unit - frames[f].base_a;
        band = (frames[f].H + frames[f].band_a - 1) / frames[f].band_a - 1 - local / frames[f].tiles_x_a;
        strip = local % frames[f].tiles_x_a;
    }
    const FrameDesc& fd = frames[f];
    const int H = fd.H, W = fd.W, in_pitch = fd.in_pitch;
    // output columns per strip: kSW - 2 Rh, or fewer when the units are
    // those of the key kernel's narrower strips (redone here on floats)
    const int OW = fd.ow_a;
    const float* __restrict__ src = fd.in;
    const int r0 = band * fd.band_a, r1 = min(r0 + fd.band_a, H);
    // Strip s reads frame columns [s OW, s OW + kSW) and writes [s OW + Rh,
    // (s + 1) OW + Rh); the first strip also writes its left halo columns,
    // which have nothing left of them but the frame's edge.
    const int sx = strip * OW;                 // frame column of strip column 0
    const int cx = sx + lane * kV;             // frame column of this lane's first column
    const bool edge = sx + kSW > W;            // strip crosses the frame's right edge
    const bool at_left = sx == 0;
    // the rows written: C's keys (off-grid values in the float map), or the
    // output at a stop before step 5 (held in registers: re-reading the
    // descriptor for every row measured 3 % slower)
    float* const dst0 = (stop == kStopFull ? fd.c : fd.out) + cx;
    unsigned short* const kdst0 = stop == kStopFull ? fd.ck + cx : nullptr;
    const size_t dst_pitch = stop == kStopFull ? (size_t)fd.c_pitch : (size_t)fd.out_pitch;
    bool col_in[kV], col_out[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        const int c = cx + v, j = lane * kV + v;
        col_in[v] = c < W;
        col_out[v] = col_in[v] && (j >= Rh || at_left) && j < Rh + OW;
    }
    // a lane writes its four keys by one 8-byte store, or two 4-byte ones
    // (cx is even: strips start at even columns), unless some of its columns
    // are halo or beyond the frame
    bool all_out = true;
#pragma unroll
    for (int v = 0; v < kV; ++v) all_out = all_out && col_out[v];
    const bool al8 = (cx & 3) == 0;

    FirstDilation<S> s2;
    Square5<true> s3d;
    Square5<false> s3e;
    Fill7 s4;
    s2.init();
    s3d.init(ninf());
    s3e.init(pinf());
    s4.init();
    int top_row[kV];
    unsigned top_key[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        top_row[v] = INT_MAX;
        top_key[v] = 0u;
    }
    bool tops_pending = (stop == kStopFull);

    const int t0 = r0 - Rh;
    const int nsteps = (r1 - r0) + 2 * Rh;
    float raw[4][kV];
    auto load_row = [&](int t, float (&d)[kV]) {
#pragma unroll
        for (int v = 0; v < kV; ++v) d[v] = 0.0f;
        if (t >= 0 && t < H) {
            const float* p = src + (size_t)t * in_pitch + cx;
#pragma unroll
            for (int v = 0; v < kV; ++v)
                if (col_in[v]) d[v] = __ldcs(p + v);
        }
    };
#pragma unroll
    for (int q = 0; q < 4; ++q) load_row(t0 + q, raw[q]);

    // Consecutive in-frame input rows with no valid depth.  Every value in the
    // rings depends on the last 2 * Rh + 2 input rows at most, so once more
    // than kQuiet such rows have streamed by, the rings hold exactly what an
    // all-empty history gives (0 on in-frame columns) and an empty row leaves
    // them unchanged: its outputs are 0 and its arithmetic can be skipped.
    constexpr int kQuiet = 2 * Rh + 4;
    int quiet = 0;

    auto step = [&](auto phi, int u0) {
        constexpr int PHI = decltype(phi)::value;
        const int t = t0 + u0 + PHI;
        const bool row_in = t >= 0 && t < H;
        bool mine_empty = true;
#pragma unroll
        for (int v = 0; v < kV; ++v) mine_empty &= is_empty(raw[PHI][v]);
        quiet = (row_in && __all_sync(0xffffffffu, mine_empty)) ? quiet + 1 : 0;
        if (quiet > kQuiet) {
            load_row(t + 4, raw[PHI]);
            const int r = stop == kStopInvert ? t
                        : stop == kStopDilate ? t - R1
                        : stop == kStopClose  ? t - R1 - 4
                                              : t - Rh;
            if (r >= r0 && r < r1) {
                if (stop == kStopFull) {  // C: key 0
                    unsigned short* kd = kdst0 + (size_t)r * dst_pitch;
                    if (all_out && al8) {
                        *reinterpret_cast<uint2*>(kd) = make_uint2(0u, 0u);
                    } else {
#pragma unroll
                        for (int v = 0; v < kV; ++v)
                            if (col_out[v]) kd[v] = 0;
                    }
                } else {
                    float* dst = dst0 + (size_t)r * dst_pitch;
#pragma unroll
                    for (int v = 0; v < kV; ++v)
                        if (col_out[v]) dst[v] = 0.0f;
                }
            }
            return;
        }
        // step 1
        Row x;
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const float d = raw[PHI][v];
            x.v[v] = (d >= kEmptyBelow) ? __fsub_rn(kInvertFrom, d) : 0.0f;
        }
        // out-of-frame pixels take the neutral value; the tests are
        // warp-uniform and false for inner strips away from the frame's ends
        if (!row_in || edge)
#pragma unroll
            for (int v = 0; v < kV; ++v)
                if (!row_in || !col_in[v]) x.v[v] = ninf();
        load_row(t + 4, raw[PHI]);
        // step 2: row t -> A(t - R1)
        Row a;
        s2.template push<PHI>(x, a.v, at_left);
        const int ra = t - R1;
        const bool a_in = ra >= 0 && ra < H;
        if (!a_in || edge)
#pragma unroll
            for (int v = 0; v < kV; ++v)
                if (!a_in || !col_in[v]) a.v[v] = ninf();
        // step 3, dilation: A(ra) -> D(ra - 2)
        Row dd;
        s3d.template push<PHI>(a, dd.v, at_left);
        const int rd = ra - 2;
        const bool d_in = rd >= 0 && rd < H;
        if (!d_in || edge)
#pragma unroll
            for (int v = 0; v < kV; ++v)
                if (!d_in || !col_in[v]) dd.v[v] = pinf();
        // step 3, erosion: D(rd) -> B(rd - 2)
        Row b;
        s3e.template push<PHI>(dd, b.v, at_left);
        const int rb = rd - 2;
        const bool b_in = rb >= 0 && rb < H;
        if (!b_in || edge)
#pragma unroll
            for (int v = 0; v < kV; ++v)
                if (!b_in || !col_in[v]) b.v[v] = ninf();
        // step 4: B(rb) -> C(rb - 3)
        float c[kV];
        s4.template push<PHI>(b, c, at_left);
        const int rc = rb - 3;  // == t - Rh
        if (stop == kStopFull) {
            if (rc >= r0 && rc < r1) {
                unsigned k[kV];
                bool grid = true;
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    bool ok = true;
                    k[v] = key_of(c[v], ok);
                    if (!ok) k[v] = kKeyOff;
                    grid = grid && ok;
                }
                unsigned short* kd = kdst0 + (size_t)rc * dst_pitch;
                if (all_out) {
                    const unsigned w0 = __byte_perm(k[0], k[1], 0x5410), w1 = __byte_perm(k[2], k[3], 0x5410);
                    if (al8) {
                        *reinterpret_cast<uint2*>(kd) = make_uint2(w0, w1);
                    } else {
                        reinterpret_cast<unsigned*>(kd)[0] = w0;
                        reinterpret_cast<unsigned*>(kd)[1] = w1;
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < kV; ++v)
                        if (col_out[v]) kd[v] = (unsigned short)k[v];
                }
                if (!grid) {  // values off the key grid, by value
                    float* dst = dst0 + (size_t)rc * dst_pitch;
#pragma unroll
                    for (int v = 0; v < kV; ++v)
                        if (col_out[v] && k[v] == kKeyOff) dst[v] = c[v];
                }
                if (tops_pending) {
                    bool left = false;
#pragma unroll
                    for (int v = 0; v < kV; ++v) {
                        if (col_out[v] && !is_empty(c[v]) && top_row[v] == INT_MAX) {
                            top_row[v] = rc;
                            top_key[v] = k[v];
                        }
                        left |= col_out[v] && top_row[v] == INT_MAX;
                    }
                    tops_pending = __any_sync(0xffffffffu, left);
                }
            }
        } else {
            // a stop before step 5: the requested map, row by row, to the output
            int r = rc;
            float val[kV];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                val[v] = c[v];
                if (stop == kStopInvert) val[v] = x.v[v];
                if (stop == kStopDilate) val[v] = a.v[v];
                if (stop == kStopClose) val[v] = b.v[v];
            }
            if (stop == kStopInvert) r = t;
            if (stop == kStopDilate) r = ra;
            if (stop == kStopClose) r = rb;
            if (r >= r0 && r < r1) {
                float* dst = dst0 + (size_t)r * dst_pitch;
#pragma unroll
                for (int v = 0; v < kV; ++v)
                    if (col_out[v]) dst[v] = val[v];
            }
        }
    };

    for (int u0 = 0; u0 < nsteps; u0 += 4) {
        step(std::integral_constant<int, 0>{}, u0);
        step(std::integral_constant<int, 1>{}, u0);
        step(std::integral_constant<int, 2>{}, u0);
        step(std::integral_constant<int, 3>{}, u0);
    }
    if (stop == kStopFull) {
#pragma unroll
        for (int v = 0; v < kV; ++v)
            if (col_out[v] && top_row[v] != INT_MAX) atomicMin(&fd.top[cx + v], top_pack(top_row[v], top_key[v]));
    }
}

}  // namespace afloat
}  // namespace
}  // namespace dcgb
