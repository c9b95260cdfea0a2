// stage_a_keys.cu -- steps 1-4 of arXiv 1802.00036, Section IV, on packed
// 16-bit keys.
//
// The same streaming design as stage_a.cu (one warp per column strip x row
// band, register rings for every vertical window, the horizontal part from
// the lane's own columns and its neighbours' by warp shuffles), on the
// values' 16-bit keys: an inverted depth v = 100 - d with d on KITTI's grid
// of 1/256 m is k / 256 for an integer k <= 25600, and the key k orders
// exactly as v does, so every maximum and minimum of steps 2-4 is the
// maximum or minimum of keys.  A lane's four columns are two 32-bit words of
// two keys each; one 3-input packed min or max (vimnmx3 on u16x2) handles
// two columns, and the pairs shifted by one column are byte permutes of
// adjacent words.  Empty pixels and pixels outside the frame hold key 0 (no
// valid key is smaller) before a maximum, 0xFFFF before a minimum.
//
// Step 1 turns each input depth into its key as the row arrives; a unit
// with an input off the grid (a valid depth, or an empty one between 0 and
// 0.1 m) or a depth above 100 m (whose inversion is negative) is appended to
// the float unit of stage_a_float.cuh, which the same warp runs at once:
// it writes the whole unit again.  C's
// rows go out as the words themselves, the tops by the same 64-bit
// atomicMin as there.  Only the full chain (stop == kStopFull) runs here.
#include "stage_a_float.cuh"

#include <climits>
#include <type_traits>

namespace dcgb {
namespace {

// kP key words (2 kP columns) per lane: strips of 64 kP columns.

constexpr unsigned kNeutralMax = 0u;           // before a maximum: no key is smaller
constexpr unsigned kNeutralMin = 0xFFFFFFFFu;  // before a minimum: no key is larger

template <bool kMax>
__device__ __forceinline__ unsigned ext3(unsigned a, unsigned b, unsigned c)
{
    return kMax ? __vimax3_u16x2(a, b, c) : __vimin3_u16x2(a, b, c);
}

// A row of a lane: w[2 .. 2 + kP) its own words (columns 0-1, 2-3, ..),
// w[0], w[1] the two words left of them (columns -4..-1), w[2 + kP],
// w[3 + kP] the two right of them.  Word i holds columns (2i - 4, 2i - 3).
template <int kP>
struct KRow {
    unsigned w[kP + 4];
    // Columns (2i - 3, 2i - 2): the pair shifted by one column.
    __device__ __forceinline__ unsigned shifted(int i) const { return __byte_perm(w[i], w[i + 1], 0x5432); }
    // fetch the neighbour words for radius R (1..3); at the frame's left
    // edge (at_left) those left of the strip are the neutral value
    template <int R>
    __device__ __forceinline__ void neighbours(bool at_left, unsigned neutral)
    {
        const int lane = threadIdx.x & 31;
        if (kP >= 2) {
            w[1] = __shfl_up_sync(0xffffffffu, w[kP + 1], 1);
            w[kP + 2] = __shfl_down_sync(0xffffffffu, w[2], 1);
            if (R >= 3) {
                w[0] = __shfl_up_sync(0xffffffffu, w[kP], 1);
                w[kP + 3] = __shfl_down_sync(0xffffffffu, w[3], 1);
            }
            if (at_left && lane == 0) {
                w[1] = neutral;
                if (R >= 3) w[0] = neutral;
            }
        } else {
            w[1] = __shfl_up_sync(0xffffffffu, w[2], 1);
            w[3] = __shfl_down_sync(0xffffffffu, w[2], 1);
            if (R >= 3) {
                w[0] = __shfl_up_sync(0xffffffffu, w[2], 2);
                w[4] = __shfl_down_sync(0xffffffffu, w[2], 2);
            }
            if (at_left && lane == 0) w[1] = neutral;
            if (R >= 3 && at_left && lane < 2) w[0] = neutral;
        }
    }
};

// Horizontal extremes of radius 1, 2, 3 for the lane's pair j (columns 2j,
// 2j + 1): h1 over [-1, 1], h2 over [-2, 2], h3 over [-3, 3].
template <bool kMax, int kP>
__device__ __forceinline__ unsigned hext1(const KRow<kP>& x, int j)
{
    return ext3<kMax>(x.shifted(1 + j), x.w[2 + j], x.shifted(2 + j));
}
template <bool kMax, int kP>
__device__ __forceinline__ unsigned hext2(const KRow<kP>& x, int j, unsigned h1)
{
    return ext3<kMax>(h1, x.w[1 + j], x.w[3 + j]);
}
template <bool kMax, int kP>
__device__ __forceinline__ unsigned hext3(const KRow<kP>& x, int j, unsigned h2)
{
    return ext3<kMax>(h2, x.shifted(j), x.shifted(3 + j));
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
template <bool kMax, int kP>
struct Window7 {
    unsigned h[2][kP], u[4][kP];
    __device__ void init(unsigned fill)
    {
        for (int v = 0; v < kP; ++v) {
            h[0][v] = h[1][v] = fill;
            u[0][v] = u[1][v] = u[2][v] = u[3][v] = fill;
        }
    }
    template <int PHI>
    __device__ __forceinline__ unsigned push(int v, unsigned hn)
    {
        const unsigned un = ext3<kMax>(h[PHI & 1][v], h[(PHI + 1) & 1][v], hn);
        const unsigned o = ext3<kMax>(u[PHI & 3][v], u[(PHI + 3) & 3][v], hn);
        h[PHI & 1][v] = hn;
        u[PHI & 3][v] = un;
        return o;
    }
};

// Step 2 for each element (the rows of Fig. 4's shapes as horizontal
// extremes of radius 0..3): push() takes input row t and returns the
// dilation of row t - r1, exactly as the float rings of stage_a.cu.
template <int S, int kP> struct FirstDilation;

template <int kP> struct FirstDilation<kDiamond5, kP> {
    unsigned x[2][kP], p[2][kP], h1[kP];
    __device__ void init()
    {
        for (int v = 0; v < kP; ++v) x[0][v] = x[1][v] = p[0][v] = p[1][v] = h1[v] = kNeutralMax;
    }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<2>(at_left, kNeutralMax);
#pragma unroll
        for (int v = 0; v < kP; ++v) {
            const unsigned a1 = hext1<true>(in, v);
            const unsigned a2 = hext2<true>(in, v, a1);
            const unsigned pn = ext3<true>(x[PHI & 1][v], h1[v], a2);
            out[v] = ext3<true>(p[PHI & 1][v], h1[v], in.w[2 + v]);
            x[PHI & 1][v] = in.w[2 + v];
            p[PHI & 1][v] = pn;
            h1[v] = a1;
        }
    }
};

template <int kP> struct FirstDilation<kFull5, kP> {
    unsigned h[2][kP], s[2][kP];
    __device__ void init()
    {
        for (int v = 0; v < kP; ++v) h[0][v] = h[1][v] = s[0][v] = s[1][v] = kNeutralMax;
    }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<2>(at_left, kNeutralMax);
#pragma unroll
        for (int v = 0; v < kP; ++v) {
            const unsigned a2 = hext2<true>(in, v, hext1<true>(in, v));
            const unsigned hm1 = h[(PHI + 1) & 1][v], hm2 = h[PHI & 1][v];
            out[v] = ext3<true>(s[PHI & 1][v], hm1, a2);
            s[PHI & 1][v] = ext3<true>(hm2, hm1, a2);
            h[PHI & 1][v] = a2;
        }
    }
};

template <int kP> struct FirstDilation<kCross5, kP> {
    unsigned x[2][kP], p[2][kP];
    __device__ void init()
    {
        for (int v = 0; v < kP; ++v) x[0][v] = x[1][v] = p[0][v] = p[1][v] = kNeutralMax;
    }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<2>(at_left, kNeutralMax);
#pragma unroll
        for (int v = 0; v < kP; ++v) {
            const unsigned a2 = hext2<true>(in, v, hext1<true>(in, v));
            const unsigned xm1 = x[(PHI + 1) & 1][v], xm2 = x[PHI & 1][v];
            const unsigned pn = ext3<true>(xm2, xm1, a2);
            out[v] = ext3<true>(p[PHI & 1][v], xm1, in.w[2 + v]);
            x[PHI & 1][v] = in.w[2 + v];
            p[PHI & 1][v] = pn;
        }
    }
};

template <int kP> struct FirstDilation<kFull3, kP> {
    unsigned h[2][kP];
    __device__ void init()
    {
        for (int v = 0; v < kP; ++v) h[0][v] = h[1][v] = kNeutralMax;
    }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<1>(at_left, kNeutralMax);
#pragma unroll
        for (int v = 0; v < kP; ++v) {
            const unsigned a1 = hext1<true>(in, v);
            out[v] = ext3<true>(h[PHI & 1][v], h[(PHI + 1) & 1][v], a1);
            h[PHI & 1][v] = a1;
        }
    }
};

template <int kP> struct FirstDilation<kCircle5, kP> {
    unsigned h1[2][kP], h2[kP], p[2][kP];
    __device__ void init()
    {
        for (int v = 0; v < kP; ++v) h1[0][v] = h1[1][v] = h2[v] = p[0][v] = p[1][v] = kNeutralMax;
    }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<2>(at_left, kNeutralMax);
#pragma unroll
        for (int v = 0; v < kP; ++v) {
            const unsigned a1 = hext1<true>(in, v);
            const unsigned a2 = hext2<true>(in, v, a1);
            const unsigned pn = ext3<true>(h1[PHI & 1][v], h2[v], a2);
            out[v] = ext3<true>(p[PHI & 1][v], h2[v], a1);
            h1[PHI & 1][v] = a1;
            h2[v] = a2;
            p[PHI & 1][v] = pn;
        }
    }
};

template <int kP> struct FirstDilation<kFull7, kP> {
    Window7<true, kP> w;
    __device__ void init() { w.init(kNeutralMax); }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<3>(at_left, kNeutralMax);
#pragma unroll
        for (int v = 0; v < kP; ++v)
            out[v] = w.template push<PHI>(v, hext3<true>(in, v, hext2<true>(in, v, hext1<true>(in, v))));
    }
};

// 5x5 square max or min (step 3).
template <bool kMax, int kP>
struct Square5 {
    unsigned h[2][kP], s[2][kP];
    __device__ void init(unsigned fill)
    {
        for (int v = 0; v < kP; ++v) h[0][v] = h[1][v] = s[0][v] = s[1][v] = fill;
    }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<2>(at_left, kMax ? kNeutralMax : kNeutralMin);
#pragma unroll
        for (int v = 0; v < kP; ++v) {
            const unsigned hn = hext2<kMax>(in, v, hext1<kMax>(in, v));
            const unsigned hm1 = h[(PHI + 1) & 1][v], hm2 = h[PHI & 1][v];
            out[v] = ext3<kMax>(s[PHI & 1][v], hm1, hn);
            s[PHI & 1][v] = ext3<kMax>(hm2, hm1, hn);
            h[PHI & 1][v] = hn;
        }
    }
};

// Per-key mask of the non-empty keys (> 25, i.e. values >= 0.1) of a word:
// 0xFFFF in each half that holds one.  Keys are below 0x8000, so adding
// 0x8000 - 26 to each half sets its top bit exactly when the key is >= 26,
// with no carry into the other half; a byte permute spreads the two top
// bits over their halves.
__device__ __forceinline__ unsigned nonempty_mask(unsigned w)
{
    unsigned m;
    // selector nibbles 9 and B: the sign of byte 1 (bit 15) and of byte 3
    // (bit 31), replicated over the byte (prmt's sign mode)
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(m) : "r"(w + 0x7FE67FE6u));
    return m;
}

// Step 4: 7x7 max written into empty pixels of B only.
template <int kP>
struct Fill7 {
    Window7<true, kP> w;
    unsigned b[4][kP];  // B rows, to select C(o - 3)
    __device__ void init()
    {
        w.init(kNeutralMax);
        for (int v = 0; v < kP; ++v) b[0][v] = b[1][v] = b[2][v] = b[3][v] = kNeutralMax;
    }
    template <int PHI>
    __device__ __forceinline__ void push(KRow<kP>& in, unsigned* out, bool at_left)
    {
        in.template neighbours<3>(at_left, kNeutralMax);
#pragma unroll
        for (int v = 0; v < kP; ++v) {
            const unsigned hn = hext3<true>(in, v, hext2<true>(in, v, hext1<true>(in, v)));
            const unsigned m7 = w.template push<PHI>(v, hn);
            const unsigned bc = b[(PHI + 1) & 3][v];  // B(o - 3)
            const unsigned keep = nonempty_mask(bc);
            out[v] = (bc & keep) | (m7 & ~keep);
            b[PHI & 3][v] = in.w[2 + v];
        }
    }
};

// Step 1 for two columns: the keys of their inverted depths, packed (the
// first in the low half).  A depth d >= 0.1 on the 1/256 m grid and at most
// 100 m has the key 25600 - 256 d; an empty one (below 0.1, negative or
// NaN) has key 0.  With v = max(d, 0) (0 for NaN), f = 2^23 + 25600 - 256 v
// is exact, its low 16 bits the key, when 256 v is an integer no larger
// than 25600; r = 256 v - (2^23 + 25600 - f) is then exactly +0 (r's bits
// are OR-ed into racc) and f >= 2^23 exactly when v <= 100 (f's minimum
// goes to fmn): a unit whose racc is not 0 or whose fmn is below 2^23 is
// off the key grid.  Keys >= 25575 (v <= 25/256, below 0.1) are the empty
// ones: adding 0x8000 - 25575 to each half sets its top bit exactly then,
// with no carry out of the half (keys are at most 25600 here), and prmt's
// sign mode spreads the two bits into a mask of the halves to clear.  The
// arithmetic is three FMA-pipe operations per depth.
__device__ __forceinline__ unsigned input_word(float d0, float d1, unsigned& racc, float& fmn)
{
    const float v0 = fmaxf(d0, 0.0f), v1 = fmaxf(d1, 0.0f);
    const float f0 = fmaf(-v0, 256.0f, 8414208.0f), f1 = fmaf(-v1, 256.0f, 8414208.0f);  // 2^23 + 25600
    const float r0 = fmaf(v0, 256.0f, f0 - 8414208.0f), r1 = fmaf(v1, 256.0f, f1 - 8414208.0f);
    racc |= __float_as_uint(r0) | __float_as_uint(r1);
    fmn = fminf(fmn, fminf(f0, f1));
    const unsigned w = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x5410);
    unsigned e;
    // selector nibbles 9 and B: the signs of bytes 1 and 3, over their halves
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(e) : "r"(w + 0x1C191C19u));
    return w & ~e;
}

// One unit of steps 1-4 on keys; false if its inputs left the key grid
// (then the float kernel redoes it: no top has been written).  kP words
// (2 kP columns) per lane: a strip of 64 kP columns, of which the frame's
// ow_a output columns start Rh in.
template <int S, int kP>
__device__ __forceinline__ bool keys_unit(const FrameDesc* __restrict__ frames, int n_frames, int unit,
                                          int band_stride)
{
    constexpr int kV = 2 * kP;        // columns per lane
    constexpr int kSW = 32 * kV;      // strip width in columns
    constexpr int R1 = ShapeInfo<S>::r;
    constexpr int Rh = R1 + 7;        // halo, horizontal and vertical
    const int lane = threadIdx.x & 31;
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
    const int H = fd.H, W = fd.W, in_pitch = fd.in_pitch, OW = fd.ow_a;
    const float* __restrict__ src = fd.in;
    const int r0 = band * fd.band_a, r1 = min(r0 + fd.band_a, H);
    const int sx = strip * OW;
    const int cx = sx + lane * kV;
    const bool edge = sx + kSW > W;
    const bool at_left = sx == 0;
    unsigned short* const kdst0 = fd.ck + cx;
    const size_t pitch = (size_t)fd.c_pitch;
    bool col_in[kV], col_out[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        const int c = cx + v, j = lane * kV + v;
        col_in[v] = c < W;
        col_out[v] = col_in[v] && (j >= Rh || at_left) && j < Rh + OW;
    }
    bool all_out = true;
#pragma unroll
    for (int v = 0; v < kV; ++v) all_out = all_out && col_out[v];
    const bool al8 = (cx & 3) == 0;
    // in-frame halves of the lane's words (edge strips only)
    unsigned in_mask[kP];
#pragma unroll
    for (int v = 0; v < kP; ++v)
        in_mask[v] = (col_in[2 * v] ? 0xFFFFu : 0u) | (col_in[2 * v + 1] ? 0xFFFF0000u : 0u);

    FirstDilation<S, kP> s2;
    Square5<true, kP> s3d;
    Square5<false, kP> s3e;
    Fill7<kP> s4;
    s2.init();
    s3d.init(kNeutralMax);
    s3e.init(kNeutralMin);
    s4.init();
    int top_row[kV];
    unsigned top_key[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        top_row[v] = INT_MAX;
        top_key[v] = 0u;
    }
    bool tops_pending = true;
    unsigned racc = 0u;      // the bits of every r of input_word: 0 on the key grid
    float fmn = 8414208.0f;  // the smallest f of input_word: >= 2^23 for depths up to 100 m

    const int t0 = r0 - Rh;
    // every row the stages' outputs hold lies inside the frame (A rows from
    // t0 - R1, B rows down to t0 - R1 - 4, A rows up to r1 + Rh - 1 - R1):
    // the per-row frame checks below are skipped
    const bool rows_inside = t0 - R1 - 4 >= 0 && r1 + Rh - R1 <= H;
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

    // rows of C written by one store pattern: the words whole (one 8-byte or
    // 4-byte stores: cx is even, strips start at even columns), or single keys
    auto store_c = [&](int r, const unsigned* c) {
        unsigned short* kd = kdst0 + (size_t)r * pitch;
        if (all_out) {
            if (kP >= 2 && al8) {
#pragma unroll
                for (int v = 0; v + 1 < kP; v += 2) reinterpret_cast<uint2*>(kd)[v / 2] = make_uint2(c[v], c[v + 1]);
            } else {
#pragma unroll
                for (int v = 0; v < kP; ++v) reinterpret_cast<unsigned*>(kd)[v] = c[v];
            }
        } else {
#pragma unroll
            for (int v = 0; v < kV; ++v)
                if (col_out[v]) kd[v] = (unsigned short)((v & 1) ? c[v >> 1] >> 16 : c[v >> 1] & 0xFFFFu);
        }
    };

    // Consecutive in-frame input rows of zeros (empty depths): after more
    // than kQuiet of them the rings hold what an all-empty history gives and
    // such a row leaves them unchanged (outputs 0), as in stage_a.cu.
    constexpr int kQuiet = 2 * Rh + 4;
    int quiet = 0;

    auto step = [&](auto phi, int u0) {
        constexpr int PHI = decltype(phi)::value;
        const int t = t0 + u0 + PHI;
        const bool row_in = t >= 0 && t < H;
        unsigned bits = 0u;
#pragma unroll
        for (int v = 0; v < kV; ++v) bits |= __float_as_uint(raw[PHI][v]);
        quiet = (row_in && __all_sync(0xffffffffu, bits == 0u)) ? quiet + 1 : 0;
        if (quiet > kQuiet) {
            load_row(t + 4, raw[PHI]);
            const int r = t - Rh;
            const unsigned zero[kP] = {};
            if (r >= r0 && r < r1) store_c(r, zero);
            return;
        }
        // step 1: the keys of the inverted depths; rows and columns outside the
        // frame were loaded as 0, whose key is the neutral 0
        KRow<kP> x;
#pragma unroll
        for (int v = 0; v < kP; ++v) x.w[2 + v] = input_word(raw[PHI][2 * v], raw[PHI][2 * v + 1], racc, fmn);
        load_row(t + 4, raw[PHI]);
        // step 2: row t -> A(t - R1)
        KRow<kP> a;
        s2.template push<PHI>(x, a.w + 2, at_left);
        const int ra = t - R1;
        if (!rows_inside && (ra < 0 || ra >= H)) {
#pragma unroll
            for (int v = 0; v < kP; ++v) a.w[2 + v] = kNeutralMax;
        } else if (edge) {
#pragma unroll
            for (int v = 0; v < kP; ++v) a.w[2 + v] &= in_mask[v];
        }
        // step 3, dilation: A(ra) -> D(ra - 2)
        KRow<kP> dd;
        s3d.template push<PHI>(a, dd.w + 2, at_left);
        const int rd = ra - 2;
        if (!rows_inside && (rd < 0 || rd >= H)) {
#pragma unroll
            for (int v = 0; v < kP; ++v) dd.w[2 + v] = kNeutralMin;
        } else if (edge) {
#pragma unroll
            for (int v = 0; v < kP; ++v) dd.w[2 + v] |= ~in_mask[v];
        }
        // step 3, erosion: D(rd) -> B(rd - 2)
        KRow<kP> b;
        s3e.template push<PHI>(dd, b.w + 2, at_left);
        const int rb = rd - 2;
        if (!rows_inside && (rb < 0 || rb >= H)) {
#pragma unroll
            for (int v = 0; v < kP; ++v) b.w[2 + v] = kNeutralMax;
        } else if (edge) {
#pragma unroll
            for (int v = 0; v < kP; ++v) b.w[2 + v] &= in_mask[v];
        }
        // step 4: B(rb) -> C(rb - 3)
        unsigned c[kP];
        s4.template push<PHI>(b, c, at_left);
        const int rc = rb - 3;  // == t - Rh
        if (rc >= r0 && rc < r1) {
            store_c(rc, c);
            if (tops_pending) {
                bool left = false;
#pragma unroll
                for (int v = 0; v < kV; ++v) {
                    const unsigned k = (v & 1) ? c[v >> 1] >> 16 : c[v >> 1] & 0xFFFFu;
                    if (col_out[v] && k > kEmptyKeyMax && top_row[v] == INT_MAX) {
                        top_row[v] = rc;
                        top_key[v] = k;
                    }
                    left |= col_out[v] && top_row[v] == INT_MAX;
                }
                tops_pending = __any_sync(0xffffffffu, left);
            }
        }
    };

    for (int u0 = 0; u0 < nsteps; u0 += 4) {
        step(std::integral_constant<int, 0>{}, u0);
        step(std::integral_constant<int, 1>{}, u0);
        step(std::integral_constant<int, 2>{}, u0);
        step(std::integral_constant<int, 3>{}, u0);
        // inputs off the key grid: the float kernel redoes the whole unit, so
        // stop at once (one vote per four rows)
        if (__any_sync(0xffffffffu, racc != 0u || fmn < 8388608.0f)) return false;
    }
#pragma unroll
    for (int v = 0; v < kV; ++v)
        if (col_out[v] && top_row[v] != INT_MAX) atomicMin(&fd.top[cx + v], top_pack(top_row[v], top_key[v]));
    return true;
}

// Persistent, as stage_a_stream: warp w starts with unit w, then takes the
// next unclaimed unit from work[2]; unit 0 zeroes work[0] and work[1] for
// stage B.  A unit whose inputs are off the key grid is done again on
// floats by the same warp (the float unit needs more registers than this
// kernel's 128: it spills, on a path that KITTI's 1/256 m depths never
// take).
template <int S, int kP>
__global__ void __launch_bounds__(kThreadsA, kStageAKeysWarpsPerSM)
stage_a_keys(const FrameDesc* __restrict__ frames, int n_frames, int total_units, int* __restrict__ work,
             int band_stride)
{
    wait_previous_kernel();  // the frame table, the reset tops and counters
    allow_next_kernel();
    const int lane = threadIdx.x & 31;
    int unit = blockIdx.x * (kThreadsA / 32) + (threadIdx.x >> 5);
    if (unit == 0 && lane < 2) work[lane] = 0;  // step-6 count, stage-B tile counter
    const int warps = gridDim.x * (kThreadsA / 32);
    while (unit < total_units) {  // whole warps only
        if (!keys_unit<S, kP>(frames, n_frames, unit, band_stride))
            afloat::stage_a_unit<S>(frames, n_frames, unit, kStopFull, band_stride);
        int next = 0;
        if (lane == 0) next = atomicAdd(work + 2, 1);
        unit = warps + __shfl_sync(0xffffffffu, next, 0);
    }
}

template <int S, int kP>
cudaError_t launch_shape(const FrameDesc* d_frames, int n_frames, int total_units, int* work, int band_stride,
                         int sm_count, cudaStream_t stream)
{
    const int per_block = kThreadsA / 32;
    int grid = (total_units + per_block - 1) / per_block;
    if (grid > kStageAKeysWarpsPerSM * sm_count) grid = kStageAKeysWarpsPerSM * sm_count;  // persistent
    if (grid < 1) return cudaSuccess;
    return launch_after_previous(stage_a_keys<S, kP>, dim3(grid), dim3(kThreadsA), 0, stream, d_frames, n_frames,
                                 total_units, work, band_stride);
}

template <int kP>
cudaError_t launch_words(const FrameDesc* d_frames, int n_frames, int total_units, int shape, int* work,
                         int band_stride, int sm_count, cudaStream_t stream)
{
    switch (shape) {
    case kDiamond5: return launch_shape<kDiamond5, kP>(d_frames, n_frames, total_units, work, band_stride, sm_count, stream);
    case kFull5: return launch_shape<kFull5, kP>(d_frames, n_frames, total_units, work, band_stride, sm_count, stream);
    case kCross5: return launch_shape<kCross5, kP>(d_frames, n_frames, total_units, work, band_stride, sm_count, stream);
    case kFull3: return launch_shape<kFull3, kP>(d_frames, n_frames, total_units, work, band_stride, sm_count, stream);
    case kCircle5: return launch_shape<kCircle5, kP>(d_frames, n_frames, total_units, work, band_stride, sm_count, stream);
    case kFull7: return launch_shape<kFull7, kP>(d_frames, n_frames, total_units, work, band_stride, sm_count, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

namespace {
template <int kP>
cudaError_t preload_words()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, stage_a_keys<kDiamond5, kP>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_keys<kFull5, kP>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_keys<kCross5, kP>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_keys<kFull3, kP>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_keys<kCircle5, kP>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, stage_a_keys<kFull7, kP>);
    return e;
}
}  // namespace

cudaError_t preload_stage_a_keys()
{
    const cudaError_t e = preload_words<1>();
    return e == cudaSuccess ? preload_words<2>() : e;
}

cudaError_t launch_stage_a_keys(const FrameDesc* d_frames, int n_frames, int total_units, int shape, int strip_cols,
                                int* work, int band_stride, int sm_count, cudaStream_t stream)
{
    if (strip_cols == 64)
        return launch_words<1>(d_frames, n_frames, total_units, shape, work, band_stride, sm_count, stream);
    if (strip_cols == 128)
        return launch_words<2>(d_frames, n_frames, total_units, shape, work, band_stride, sm_count, stream);

    return cudaErrorInvalidValue;
}

}  // namespace dcgb
