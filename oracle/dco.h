/*
 * dco.h -- CPU oracle for the classical depth-completion chain of
 * Ku, Harakeh, Waslander, "In Defense of Classical Image Processing: Fast
 * Depth Completion on the CPU" (arXiv 1802.00036), Section IV, steps 1-8.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, literal statement of
 * what the method computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The GPU library shares no
 * code, header, table or constant with it.
 *
 * Every map is a row-major, densely packed H x W array of float (the depth
 * maps of the method are float32 images).  Arithmetic that is not a pure
 * selection (inversion, Gaussian and bilateral sums) is done in double and
 * rounded once when stored.  Out-of-frame pixels are ignored by max and min,
 * the median replicates the border and the blurs mirror it without repeating
 * the edge pixel (reflect-101).
 */
#ifndef DCO_H
#define DCO_H

#ifdef __cplusplus
extern "C" {
#endif

/* Structuring elements (Section IV-2, Fig. 4, Table 2).  Tap sets:
 *   DIAMOND5 |dy|+|dx| <= 2 (13 taps), FULL5 5x5, CROSS5 dy==0 or dx==0
 *   within 5x5 (9 taps), FULL3 3x3, CIRCLE5 dy^2+dx^2 <= 5 (21 taps),
 *   FULL7 7x7. */
enum {
    DCO_SHAPE_DIAMOND5 = 0,
    DCO_SHAPE_FULL5 = 1,
    DCO_SHAPE_CROSS5 = 2,
    DCO_SHAPE_FULL3 = 3,
    DCO_SHAPE_CIRCLE5 = 4,
    DCO_SHAPE_FULL7 = 5
};

/* Blur after the optional median (Section IV-7, Table 3). */
enum { DCO_BLUR_NONE = 0, DCO_BLUR_GAUSS = 1, DCO_BLUR_BILATERAL = 2 };

/* Where the chain stops.  Every stop before DCO_STOP_FULL returns the map in
 * the inverted domain (valid pixels hold 100 - depth, empty pixels 0). */
enum {
    DCO_STOP_FULL = 0,       /* step 8: depth out                           */
    DCO_STOP_INVERT = 1,     /* after step 1                                */
    DCO_STOP_DILATE = 2,     /* after step 2                                */
    DCO_STOP_CLOSE = 3,      /* after step 3                                */
    DCO_STOP_FILL7 = 4,      /* after step 4                                */
    DCO_STOP_EXTEND = 5,     /* after step 5                                */
    DCO_STOP_FILL_LARGE = 6, /* after step 6                                */
    DCO_STOP_MEDIAN = 7,     /* after the median of step 7                  */
    DCO_STOP_BLUR = 8        /* after the blur of step 7 (inverted domain)  */
};

typedef struct {
    int first_kernel;    /* DCO_SHAPE_*, step 2                               */
    int large_fill;      /* odd side of the full square of step 6 (31)        */
    int median;          /* 1: 5x5 median in step 7                           */
    int blur;            /* DCO_BLUR_*, step 7                                */
    double sigma_space;  /* bilateral spatial sigma, pixels                   */
    double sigma_color;  /* bilateral range sigma, inverted metres            */
    int extend_top;      /* 1: step 5 on                                      */
    int extend_rows;     /* < 0: extend to row 0; else at most this many rows */
    int large_fill_on;   /* 1: step 6 on                                      */
    int stop_after;      /* DCO_STOP_*                                        */
} dco_params;

/* Paper defaults: diamond 5x5, 31x31 fill, median + Gaussian, full chain. */
void dco_params_default(dco_params* p);

/* Whole chain.  in and out are H x W; they must not overlap.  Returns 0, or
 * -1 on bad arguments, -2 when memory runs out. */
int dco_complete(const float* in, float* out, int H, int W, const dco_params* p);

/* The steps, exported one by one so that each can be pinned on its own. */
int dco_invert(const float* d, float* v, int H, int W);                 /* 1 */
int dco_dilate_shape(const float* a, float* o, int H, int W, int shape); /* 2 */
int dco_dilate_square(const float* a, float* o, int H, int W, int k);
int dco_erode_square(const float* a, float* o, int H, int W, int k);
int dco_close_square(const float* a, float* o, int H, int W, int k);    /* 3 */
int dco_fill_square(const float* a, float* o, int H, int W, int k);     /* 4,6 */
int dco_extend_top(const float* c, float* e, int H, int W, int max_rows); /* 5 */
int dco_median5(const float* f, float* m, int H, int W);                /* 7 */
int dco_gauss5(const float* m, double* g, int H, int W);                /* 7 */
int dco_bilateral5(const float* m, double* g, int H, int W,
                   double sigma_space, double sigma_color);             /* 7 */

/* Accuracy of a depth map against ground truth (the KITTI depth-completion
 * measures of Section V, Tables 1-3; defined by the benchmark the paper cites):
 * over pixels whose ground truth is valid (>= 0.1 m),
 *   out[0] RMSE  (mm)   = 1000 sqrt(mean((p - g)^2))
 *   out[1] MAE   (mm)   = 1000 mean(|p - g|)
 *   out[2] iRMSE (1/km) = 1000 sqrt(mean((1/p - 1/g)^2))
 *   out[3] iMAE  (1/km) = 1000 mean(|1/p - 1/g|)
 *   out[4] number of valid pixels
 * with 1/p taken as 0 where the prediction is empty (< 0.1).  All four are 0
 * when no pixel is valid.  Sums in double. */
int dco_metrics(const float* pred, const float* gt, int H, int W, double out[5]);

/* LIDAR points to a sparse depth map (Section V: the benchmark projects the
 * scans into the image with the camera calibration).  Point i is
 * (xyz[3i], xyz[3i+1], xyz[3i+2]); (u, v, w) = P (x, y, z, 1) with the 3 x 4
 * row-major matrix P, in double.  A point with w > 0 lands in pixel
 * (floor(v / w), floor(u / w)) if that is inside H x W and its depth w is in
 * [d_min, d_max]; each pixel keeps its smallest depth (as float), others 0. */
int dco_project(const float* xyz, long n, const double P[12], int H, int W,
                double d_min, double d_max, float* depth);

#ifdef __cplusplus
}
#endif
#endif /* DCO_H */
