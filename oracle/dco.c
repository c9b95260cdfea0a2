/*
 * dco.c -- CPU oracle for the depth-completion chain of arXiv 1802.00036
 * (Ku, Harakeh, Waslander), Section IV, steps 1-8.
 *
 * TEST INFRASTRUCTURE ONLY: this file states what the method computes, as
 * plainly as possible, so that the GPU library can be checked against it.
 * It is single-threaded, whole-frame and step-by-step: every step reads one
 * full map and writes a fresh one, by direct loops over the structuring
 * element (no separable passes, no running-max tricks, no fusion).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - empty pixel: value < 0.1, in the raw and in the inverted domain;
 *   - steps 2 and 3 are plain grey dilation / closing of the whole map;
 *     steps 4 and 6 write only pixels that are empty before the step;
 *   - max and min ignore out-of-frame pixels, the median replicates the
 *     frame border, the Gaussian and bilateral blurs use reflect-101;
 *   - step 5 copies the topmost non-empty value of each column (after
 *     step 4) into the rows above it; an all-empty column is unchanged;
 *   - the Gaussian is the 5-tap binomial [1 4 6 4 1]/16 in each direction;
 *   - the bilateral uses the 13 offsets with dy^2 + dx^2 <= 4;
 *   - both blurs, and the final inversion, apply only where the median
 *     output is non-empty; elsewhere the output is 0.
 */
#include "dco.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define EMPTY_BELOW 0.1     /* Section IV-1: empty pixels hold 0 */
#define INVERT_FROM 100.0   /* Section IV-1 and IV-8: D_inv = 100 - D */

static int is_empty(float v) { return !((double)v >= EMPTY_BELOW); }

static int bad_dims(int H, int W) { return H < 1 || W < 1; }

void dco_params_default(dco_params* p)
{
    p->first_kernel = DCO_SHAPE_DIAMOND5;
    p->large_fill = 31;
    p->median = 1;
    p->blur = DCO_BLUR_GAUSS;
    p->sigma_space = 1.5;
    p->sigma_color = 0.5;
    p->extend_top = 1;
    p->extend_rows = -1;
    p->large_fill_on = 1;
    p->stop_after = DCO_STOP_FULL;
}

/* ---- structuring elements (Section IV-2, Fig. 4) ------------------------ */

/* Half-width of the element's bounding square, or -1 for an unknown shape. */
static int shape_radius(int shape)
{
    switch (shape) {
    case DCO_SHAPE_DIAMOND5: case DCO_SHAPE_FULL5:
    case DCO_SHAPE_CROSS5: case DCO_SHAPE_CIRCLE5: return 2;
    case DCO_SHAPE_FULL3: return 1;
    case DCO_SHAPE_FULL7: return 3;
    default: return -1;
    }
}

/* Is offset (dy, dx) part of the element? */
static int shape_has(int shape, int dy, int dx)
{
    int ay = abs(dy), ax = abs(dx);
    switch (shape) {
    case DCO_SHAPE_DIAMOND5: return ay + ax <= 2;
    case DCO_SHAPE_FULL5: return ay <= 2 && ax <= 2;
    case DCO_SHAPE_CROSS5: return (ay == 0 && ax <= 2) || (ax == 0 && ay <= 2);
    case DCO_SHAPE_FULL3: return ay <= 1 && ax <= 1;
    case DCO_SHAPE_CIRCLE5: return ay * ay + ax * ax <= 5;
    case DCO_SHAPE_FULL7: return ay <= 3 && ax <= 3;
    default: return 0;
    }
}

/* ---- step 1: inversion (Section IV-1) ----------------------------------- */

int dco_invert(const float* d, float* v, int H, int W)
{
    if (!d || !v || bad_dims(H, W)) return -1;
    for (long i = 0; i < (long)H * W; ++i) {
        /* 100 - d is exact in double for a float d >= 0.1; one rounding to
         * float gives the correctly rounded float32 difference. */
        v[i] = is_empty(d[i]) ? 0.0f : (float)(INVERT_FROM - (double)d[i]);
    }
    return 0;
}

/* ---- grey morphology with out-of-frame pixels ignored ------------------- */

int dco_dilate_shape(const float* a, float* o, int H, int W, int shape)
{
    int R = shape_radius(shape);
    if (!a || !o || bad_dims(H, W) || R < 0) return -1;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            float m = a[(long)r * W + c]; /* the origin is in every element */
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    int y = r + dy, x = c + dx;
                    if (!shape_has(shape, dy, dx)) continue;
                    if (y < 0 || y >= H || x < 0 || x >= W) continue;
                    float t = a[(long)y * W + x];
                    if (t > m) m = t;
                }
            o[(long)r * W + c] = m;
        }
    return 0;
}

static int square_extreme(const float* a, float* o, int H, int W, int k, int want_max)
{
    if (!a || !o || bad_dims(H, W) || k < 1 || (k % 2) == 0) return -1;
    int R = k / 2;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            float m = a[(long)r * W + c];
            for (int y = r - R; y <= r + R; ++y) {
                if (y < 0 || y >= H) continue;
                for (int x = c - R; x <= c + R; ++x) {
                    if (x < 0 || x >= W) continue;
                    float t = a[(long)y * W + x];
                    if (want_max ? (t > m) : (t < m)) m = t;
                }
            }
            o[(long)r * W + c] = m;
        }
    return 0;
}

int dco_dilate_square(const float* a, float* o, int H, int W, int k)
{
    return square_extreme(a, o, H, W, k, 1);
}

int dco_erode_square(const float* a, float* o, int H, int W, int k)
{
    return square_extreme(a, o, H, W, k, 0);
}

/* ---- step 3: closing = dilation then erosion (Section IV-3) ------------- */

int dco_close_square(const float* a, float* o, int H, int W, int k)
{
    if (!a || !o || bad_dims(H, W)) return -1;
    float* t = (float*)malloc(sizeof(float) * (size_t)H * (size_t)W);
    if (!t) return -2;
    int rc = dco_dilate_square(a, t, H, W, k);
    if (rc == 0) rc = dco_erode_square(t, o, H, W, k);
    free(t);
    return rc;
}

/* ---- steps 4 and 6: fill empty pixels from a k x k dilation ------------- */

int dco_fill_square(const float* a, float* o, int H, int W, int k)
{
    if (!a || !o || bad_dims(H, W) || k < 1 || (k % 2) == 0) return -1;
    int R = k / 2;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            float here = a[(long)r * W + c];
            if (!is_empty(here)) { o[(long)r * W + c] = here; continue; }
            float m = here;
            for (int y = r - R; y <= r + R; ++y) {
                if (y < 0 || y >= H) continue;
                for (int x = c - R; x <= c + R; ++x) {
                    if (x < 0 || x >= W) continue;
                    float t = a[(long)y * W + x];
                    if (t > m) m = t;
                }
            }
            o[(long)r * W + c] = m;
        }
    return 0;
}

/* ---- step 5: extension to the top of the frame (Section IV-5) ---------- */

int dco_extend_top(const float* cmap, float* e, int H, int W, int max_rows)
{
    if (!cmap || !e || bad_dims(H, W)) return -1;
    memcpy(e, cmap, sizeof(float) * (size_t)H * (size_t)W);
    for (int c = 0; c < W; ++c) {
        int top = -1;
        for (int r = 0; r < H; ++r)
            if (!is_empty(cmap[(long)r * W + c])) { top = r; break; }
        if (top < 0) continue; /* no value in this column: left as it is */
        int first = 0;
        if (max_rows >= 0 && top - max_rows > 0) first = top - max_rows;
        float value = cmap[(long)top * W + c];
        for (int r = first; r < top; ++r) e[(long)r * W + c] = value;
    }
    return 0;
}

/* ---- step 7: 5x5 median, replicated border (Section IV-7) -------------- */

static int clampi(int p, int n) { return p < 0 ? 0 : (p >= n ? n - 1 : p); }

int dco_median5(const float* f, float* m, int H, int W)
{
    if (!f || !m || bad_dims(H, W)) return -1;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            float w[25];
            int n = 0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx)
                    w[n++] = f[(long)clampi(r + dy, H) * W + clampi(c + dx, W)];
            /* insertion sort of the 25 values, then take the middle one */
            for (int i = 1; i < 25; ++i) {
                float x = w[i];
                int j = i - 1;
                while (j >= 0 && w[j] > x) { w[j + 1] = w[j]; --j; }
                w[j + 1] = x;
            }
            m[(long)r * W + c] = w[12];
        }
    return 0;
}

/* ---- step 7: 5x5 Gaussian and bilateral blur, reflect-101 border -------- */

/* Mirror p into [0, n) without repeating the edge pixel: -1 -> 1, n -> n-2. */
static int reflect101(int p, int n)
{
    if (n == 1) return 0;
    while (p < 0 || p >= n) p = (p < 0) ? -p : 2 * (n - 1) - p;
    return p;
}

int dco_gauss5(const float* mm, double* g, int H, int W)
{
    static const double w[5] = {1.0, 4.0, 6.0, 4.0, 1.0}; /* binomial, sum 16 */
    if (!mm || !g || bad_dims(H, W)) return -1;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            float here = mm[(long)r * W + c];
            if (is_empty(here)) { g[(long)r * W + c] = here; continue; }
            double s = 0.0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx)
                    s += w[dy + 2] * w[dx + 2] *
                         (double)mm[(long)reflect101(r + dy, H) * W + reflect101(c + dx, W)];
            g[(long)r * W + c] = s / 256.0;
        }
    return 0;
}

int dco_bilateral5(const float* mm, double* g, int H, int W,
                   double sigma_space, double sigma_color)
{
    if (!mm || !g || bad_dims(H, W) || !(sigma_space > 0) || !(sigma_color > 0))
        return -1;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            float here = mm[(long)r * W + c];
            if (is_empty(here)) { g[(long)r * W + c] = here; continue; }
            double num = 0.0, den = 0.0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx) {
                    if (dy * dy + dx * dx > 4) continue; /* disk of radius 2 */
                    double v = mm[(long)reflect101(r + dy, H) * W + reflect101(c + dx, W)];
                    double diff = v - (double)here;
                    double ws = exp(-(double)(dy * dy + dx * dx) / (2.0 * sigma_space * sigma_space));
                    double wc = exp(-(diff * diff) / (2.0 * sigma_color * sigma_color));
                    num += v * ws * wc;
                    den += ws * wc;
                }
            g[(long)r * W + c] = num / den;
        }
    return 0;
}

/* ---- the whole chain, steps 1-8 in the paper's order -------------------- */

int dco_complete(const float* in, float* out, int H, int W, const dco_params* p)
{
    if (!in || !out || !p || bad_dims(H, W)) return -1;
    if (shape_radius(p->first_kernel) < 0) return -1;
    if (p->large_fill < 1 || (p->large_fill % 2) == 0) return -1;
    if (p->blur < DCO_BLUR_NONE || p->blur > DCO_BLUR_BILATERAL) return -1;
    if (p->stop_after < DCO_STOP_FULL || p->stop_after > DCO_STOP_BLUR) return -1;

    size_t n = (size_t)H * (size_t)W;
    float* a = (float*)malloc(sizeof(float) * n);
    float* b = (float*)malloc(sizeof(float) * n);
    double* g = (double*)malloc(sizeof(double) * n);
    int rc = (a && b && g) ? 0 : -2;
    int stop = p->stop_after;

#define STEP(call) do { if (rc == 0) rc = (call); } while (0)
#define SWAP() do { float* t_ = a; a = b; b = t_; } while (0)
    /* after every step the current map is in a */
    STEP(dco_invert(in, a, H, W));                                  /* 1 */
    if (rc == 0 && stop != DCO_STOP_INVERT) {
        STEP(dco_dilate_shape(a, b, H, W, p->first_kernel)); SWAP(); /* 2 */
    }
    if (rc == 0 && stop != DCO_STOP_INVERT && stop != DCO_STOP_DILATE) {
        STEP(dco_close_square(a, b, H, W, 5)); SWAP();              /* 3 */
    }
    if (rc == 0 && (stop == DCO_STOP_FULL || stop >= DCO_STOP_FILL7)) {
        STEP(dco_fill_square(a, b, H, W, 7)); SWAP();               /* 4 */
    }
    if (rc == 0 && (stop == DCO_STOP_FULL || stop >= DCO_STOP_EXTEND) && p->extend_top) {
        STEP(dco_extend_top(a, b, H, W, p->extend_rows)); SWAP();   /* 5 */
    }
    if (rc == 0 && (stop == DCO_STOP_FULL || stop >= DCO_STOP_FILL_LARGE) && p->large_fill_on) {
        STEP(dco_fill_square(a, b, H, W, p->large_fill)); SWAP();   /* 6 */
    }
    if (rc == 0 && (stop == DCO_STOP_FULL || stop >= DCO_STOP_MEDIAN) && p->median) {
        STEP(dco_median5(a, b, H, W)); SWAP();                      /* 7 */
    }
#undef STEP
#undef SWAP

    if (rc == 0) {
        if (stop != DCO_STOP_FULL && stop != DCO_STOP_BLUR) {
            memcpy(out, a, sizeof(float) * n);
        } else {
            /* step 7 blur, then step 8: D_out = 100 - D_inv where non-empty */
            if (p->blur == DCO_BLUR_GAUSS) rc = dco_gauss5(a, g, H, W);
            else if (p->blur == DCO_BLUR_BILATERAL)
                rc = dco_bilateral5(a, g, H, W, p->sigma_space, p->sigma_color);
            else for (size_t i = 0; i < n; ++i) g[i] = a[i];
            if (rc == 0) {
                for (size_t i = 0; i < n; ++i) {
                    if (stop == DCO_STOP_BLUR) out[i] = (float)g[i];
                    else out[i] = is_empty(a[i]) ? 0.0f : (float)(INVERT_FROM - g[i]);
                }
            }
        }
    }
    free(a);
    free(b);
    free(g);
    return rc;
}

/* ---- accuracy against ground truth (Section V, Tables 1-3) --------------- */

int dco_metrics(const float* pred, const float* gt, int H, int W, double out[5])
{
    if (!pred || !gt || !out || bad_dims(H, W)) return -1;
    double se = 0.0, ae = 0.0, ise = 0.0, iae = 0.0;
    long n = 0;
    for (long i = 0; i < (long)H * W; ++i) {
        if (is_empty(gt[i])) continue;
        const double g = gt[i], p = pred[i];
        const double ip = is_empty(pred[i]) ? 0.0 : 1.0 / p;
        const double d = p - g, id = ip - 1.0 / g;
        se += d * d;
        ae += fabs(d);
        ise += id * id;
        iae += fabs(id);
        ++n;
    }
    if (n == 0) {
        out[0] = out[1] = out[2] = out[3] = 0.0;
    } else {
        out[0] = 1000.0 * sqrt(se / n);
        out[1] = 1000.0 * (ae / n);
        out[2] = 1000.0 * sqrt(ise / n);
        out[3] = 1000.0 * (iae / n);
    }
    out[4] = (double)n;
    return 0;
}

/* ---- LIDAR points to a sparse map (Section V) ----------------------------- */

int dco_project(const float* xyz, long n, const double P[12], int H, int W,
                double d_min, double d_max, float* depth)
{
    if ((!xyz && n > 0) || !P || !depth || bad_dims(H, W) || n < 0) return -1;
    for (long i = 0; i < (long)H * W; ++i) depth[i] = 0.0f;
    for (long i = 0; i < n; ++i) {
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        const double u = P[0] * x + P[1] * y + P[2] * z + P[3];
        const double v = P[4] * x + P[5] * y + P[6] * z + P[7];
        const double w = P[8] * x + P[9] * y + P[10] * z + P[11];
        if (!(w > 0.0) || w < d_min || w > d_max) continue;
        const double col = floor(u / w), row = floor(v / w);
        if (!(col >= 0.0 && col < W && row >= 0.0 && row < H)) continue;
        const long k = (long)row * W + (long)col;
        const float d = (float)w;
        if (depth[k] == 0.0f || d < depth[k]) depth[k] = d;
    }
    return 0;
}
