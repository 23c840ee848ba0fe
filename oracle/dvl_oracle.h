/*
 * CPU oracle for the dynamic-volume-line (DVL) computation on multi-field AMR
 * data (Zellmann, Demirci, Gudukbay, "Visual Analysis of Large Multi-Field AMR
 * Data on GPUs Using Interactive Volume Lines").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, sequential, deliberately slow
 * restatement of the paper's definitions, used by the tests, by the smoke check
 * and by the benchmark's CPU-baseline leg to check and time the CUDA library.
 * The library never calls it, and the two share no code.
 *
 * Precision: integers are exact (u64 keys and widths, unsigned __int128 bin
 * arithmetic), bin sums are accumulated in double.  The per-cell quantities
 * that decide an integer (the transfer-function entry index, the fixed-point
 * width) are computed as a fixed sequence of correctly rounded float32 IEEE
 * operations, which is the precision the GPU kernels use for those decisions.
 */
#ifndef DVL_ORACLE_H
#define DVL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SFC_MORTON = 0, ORC_SFC_HILBERT = 1 };
enum { ORC_MINIMP_BEFORE_SCALE = 0, ORC_MINIMP_AFTER_POWER = 1 };
enum { ORC_VMAX_APPROX = 0, ORC_VMAX_EXACT = 1 };
enum { ORC_WIDTH_EDGE = 0, ORC_WIDTH_VOLUME = 1 };

typedef struct {
    float P;                 /* steepness exponent of Eq. 2/3 */
    float min_importance;    /* minimum importance (paper default 0.025) */
    uint32_t width;          /* plot width W in pixels (number of bins) */
    uint32_t min_imp_mode;   /* ORC_MINIMP_* */
    uint32_t vmax_mode;      /* ORC_VMAX_* */
    uint32_t width_mode;     /* ORC_WIDTH_*: scale by 2^L or by 8^L */
} orc_params;

typedef struct {
    float vmax;              /* max V used (Eq. 6 approximation or exact) */
    float inv_vmax;          /* float32 reciprocal, 0 when vmax == 0 */
    float f_upper;           /* upper bound of f over all cells */
    int32_t Q;               /* fixed-point exponent: q = rint(f * 2^Q) */
    int32_t i, j;            /* global TF index range of Eq. 5 */
    int32_t linear;          /* 1 when every width was 0 and q := 1 was used */
    int32_t pow_exact;       /* 1 when 2P is an integer in [0, 16] */
    uint64_t F;              /* sum of the fixed-point widths (Eq. 4 total) */
} orc_stats;

/* Space-filling-curve key of every cell (Sec. 2.2: cells are represented by
 * their centroid on a quantised grid).  c_d = 2*lower_d + 2^level is the
 * exact centroid in half-finest-cell units, 21 bits per axis. */
int orc_keys(uint64_t n, const int32_t* lx, const int32_t* ly, const int32_t* lz,
             const uint8_t* level, int sfc, uint64_t* keys);

/* Stable order of the cells by key (Sec. 4: the order is built once). */
int orc_order(uint64_t n, const uint64_t* keys, uint32_t* perm);

/* One DVL update over cells that are already in curve order.
 *   fields:   M arrays of n floats (field-major, fields[m*n + c])
 *   level:    n refinement levels (0 = finest)
 *   alpha:    M tables of T alpha entries (alpha[m*T + e]) in [0, 1]
 *   dom_lo/hi: transfer-function domain per field; NaN/NaN = data range
 * Outputs (each may be NULL except the bins):
 *   sum[M*W] (double), vmin/vmax/mean/y[M*W] (float), mean64[M*W], count[W],
 *   q[n], b1[n], b2[n] per cell, stats.  Returns 0, or a negative code for
 *   invalid arguments (-1) or a width bound that cannot be represented (-5). */
int orc_update(uint64_t n, uint32_t M, const float* fields, const uint8_t* level,
               uint32_t T, const float* alpha, const float* dom_lo, const float* dom_hi,
               const orc_params* prm, double* sum, float* vmin, float* vmax, float* mean,
               double* mean64, float* y, uint32_t* count, uint64_t* q, uint32_t* b1,
               uint32_t* b2, orc_stats* stats);

/* orc_update's results, bit for bit, computed on n_threads host threads
 * (OpenMP): the per-cell work is split into contiguous ranges, the Eq. 4
 * prefix is exact integer arithmetic, and each pixel is filled by one thread
 * with its cells in curve order, so no floating-point sum changes order. */
int orc_update_mt(uint64_t n, uint32_t M, const float* fields, const uint8_t* level,
                  uint32_t T, const float* alpha, const float* dom_lo, const float* dom_hi,
                  const orc_params* prm, double* sum, float* vmin, float* vmax, float* mean,
                  double* mean64, float* y, uint32_t* count, uint64_t* q, uint32_t* b1,
                  uint32_t* b2, orc_stats* stats, int n_threads);

/* orc_keys over n_threads contiguous ranges of the cells at once. */
int orc_keys_mt(uint64_t n, const int32_t* lx, const int32_t* ly, const int32_t* lz,
                const uint8_t* level, int sfc, uint64_t* keys, int n_threads);

/* Gradient of L = sum_{m,p} (abar[m][p] - target[m][p])^2 with respect to K
 * uniformly spaced alpha control points per field, where abar[m][p] is the
 * mean over the cells covering bin p of the per-cell alpha of field m, and the
 * table entry e is the linear interpolation of the control points at
 * e/(T-1).  Bin assignment and entry indices are held fixed at the values
 * of a forward update with the same inputs.  ctrl[M*K] are the parameters.
 * Writes abar[M*W] (double), grad[M*K] (double), *loss.  See orc_update for
 * the other arguments (the alpha table is built from ctrl).  With g_in
 * (M*W doubles) not NULL, grad is instead the gradient of the linear
 * functional sum_{m,p} g_in[m][p] * abar[m][p] (g_in replaces dL/dabar). */
int orc_alpha_grad(uint64_t n, uint32_t M, const float* fields, const uint8_t* level,
                   uint32_t T, uint32_t K, const float* ctrl, const float* dom_lo,
                   const float* dom_hi, const orc_params* prm, const double* target,
                   const double* g_in, double* abar, double* grad, double* loss);

/* Fixed-point widths of k sampled cells of a data set of n_total cells, one
 * by one, from the data set's global quantities (per-field data minimum and
 * maximum, deepest level) with the default TF domains and the Eq. 5/6 max V:
 * the same q as orc_update gives those cells in the whole data set (unless
 * every width of the data set is 0).  values[m*k + c], level[c]; writes q[k],
 * Q and max V.  Returns 0, -1 (arguments; exact max V is not supported) or -5. */
int orc_widths(uint64_t n_total, uint32_t M, const float* dmin, const float* dmax, uint32_t max_level, uint32_t T,
               const float* alpha, const orc_params* prm, uint64_t k, const float* values, const uint8_t* level,
               uint64_t* q, int32_t* Q_out, float* vmax_out);

/* Line-plot rasterisation of the bins (the RasterizeLines step after the
 * update, Sec. 4, Fig. 1): an H x W image, row 0 at the top, column p = bin p.
 * values[m*W + p] in [0, 1] (the bin means or their alpha) maps to the row
 *   r = clamp(floor((1 - v) * (H - 1) + 1/2), 0, H - 1)
 * in correctly rounded float32 steps.  Polyline of field m: consecutive bins
 * are joined; column p covers the rows between r_p, r_p - trunc((r_p -
 * r_{p-1}) / 2) (if p > 0) and r_p + trunc((r_{p+1} - r_p) / 2) (if p < W-1),
 * so that the two columns of a segment split its rise between them; bit m of
 * lines[row*W + p] is set where field m's line covers the pixel.  Bar plot of
 * field bar_field: bars[row*W + p] = 1 for rows r_p .. H-1, else 0.  Returns 0,
 * or -1 for invalid arguments (M in 1..8, W >= 1, H >= 1). */
int orc_rasterize(uint32_t M, uint32_t W, uint32_t H, const float* values, uint32_t bar_field,
                  uint8_t* lines, uint8_t* bars);

/* Brushing and linking (Sec. 3.5).  The cells of a pixel ROI [p0, p1] of the
 * plot are those whose span touches a pixel of it: b1[c] <= p1 and b2[c] >= p0
 * (b1, b2 from orc_update, cells in curve order).  Writes the first and last
 * such cell; returns 0, 1 if there is none, -1 for invalid arguments, -2 if
 * the set is not one contiguous run of the curve order (the mapping of Sec.
 * 3.2 is monotone, so this does not happen). */
int orc_brush(uint64_t n, const uint32_t* b1, const uint32_t* b2, uint32_t p0, uint32_t p1, uint64_t* first,
              uint64_t* last);

/* The linked selection in the 3D view (Sec. 3.5): a cell is selected when its
 * centroid's curve key lies in one of R inclusive key ranges (ranges[2r],
 * ranges[2r+1]); mask[c] = 1 for selected cells, in the order of `keys`. */
void orc_select_keys(uint64_t n, const uint64_t* keys, uint32_t R, const uint64_t* ranges, uint8_t* mask);

/* Per-field logarithmic value scale.  The paper normalises every field by its
 * own domain before the transfer function (Sec. 3.3); fields that span many
 * decades (densities, pressures) are commonly shown on a log10 axis, which
 * this transform provides before that normalisation.  A log-scaled field's
 * value v becomes log10(v), and a value <= 0 first takes the field's smallest
 * positive value.  log10 of x > 0 is evaluated as
 *   x = m * 2^e with m in [s, 2s), s = float(sqrt 2) / 2 (a subnormal x is
 *       first multiplied by 2^24, exact),
 *   z = (m - 1) / (m + 1), carried as z + dz (the quotient's residual, from
 *       fma, divided once more) so that log10 m is not limited by z's rounding,
 *   log10 m = 2 log10(e) atanh(z) = (z + dz)(c0 + c1 z^2 + ... + c4 z^8),
 *       c_k = 2 log10(e) / (2k + 1) (the Taylor series of atanh, cut where the
 *       next term is below 0.05 ulp for |z| <= 0.1716),
 *   log10 x = e * h + (e * l + log10 m), h + l = log10(2), h with 16 bits,
 * as a fixed sequence of correctly rounded float32 operations (listed in
 * orc_log10f), so that any IEEE float32 implementation of the same sequence
 * returns the same bits.  Accuracy: within 1.5 ulp of the exact log10 for
 * every positive float (checked against a float64 log10 over all of them). */
float orc_log10f(float x);

/* Replaces the n values of one field by their log10 as above, in place.
 * Returns 0, or -5 when no value is positive (the field has no log scale). */
int orc_log_field(uint64_t n, float* v);

#ifdef __cplusplus
}
#endif
#endif
