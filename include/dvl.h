/*
 * dvl.h -- C ABI of the B300-native dynamic-volume-line (DVL) library.
 *
 * Computes the 1D "interactive volume line" plot of multi-field AMR data
 * (Zellmann, Demirci, Gudukbay, "Visual Analysis of Large Multi-Field AMR
 * Data on GPUs Using Interactive Volume Lines"): cells are ordered once along
 * a space-filling curve, and on every alpha transfer-function (TF) or data
 * change each cell gets an importance-scaled width, the widths are prefix-
 * summed, and the cells are reduced into W per-pixel bins (min/max/mean).
 *
 * Conventions (all entry points):
 *   - Every call returns a dvl_status (0 = DVL_OK, negative = error); no
 *     exception, abort or trap crosses this boundary.  dvl_last_error() gives
 *     a one-line message for the last failing call on a context.
 *   - Input buffers are copied; the caller keeps ownership.  mem_kind says
 *     whether a pointer is host memory (DVL_MEM_HOST; pageable or pinned) or
 *     device memory of the context's GPU (DVL_MEM_DEVICE).
 *   - The library owns all device memory it allocates (released by
 *     dvl_destroy).  Output buffers are owned by the caller.
 *   - GPU work is issued on the context's stream, in call order.  Calls that
 *     return host-visible results (dvl_read_*, dvl_get_stats, dvl_sync)
 *     synchronise that stream; dvl_update only enqueues.
 *   - State machine: CREATED -> LOADED (dvl_load_amr) -> ORDERED
 *     (dvl_build_order).  dvl_update needs ORDERED and a TF for every field;
 *     otherwise DVL_ERR_STATE.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef DVL_H
#define DVL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dvl_ctx dvl_ctx; /* opaque, library-owned */

typedef enum {
    DVL_OK = 0,
    DVL_ERR_ARG = -1,         /* invalid argument (null, size, enum, value) */
    DVL_ERR_STATE = -2,       /* call not allowed in the current state */
    DVL_ERR_NOMEM = -3,       /* device or host allocation failed */
    DVL_ERR_CUDA = -4,        /* CUDA runtime error (incl. no usable device) */
    DVL_ERR_RANGE = -5,       /* input outside the supported domain */
    DVL_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up */
    DVL_ERR_UNSUPPORTED = -7  /* valid request this build does not support */
} dvl_status;

enum { DVL_SFC_MORTON = 0, DVL_SFC_HILBERT = 1 };
enum { DVL_MEM_HOST = 0, DVL_MEM_DEVICE = 1 };
enum { DVL_MINIMP_BEFORE_SCALE = 0, DVL_MINIMP_AFTER_POWER = 1 };
enum { DVL_VMAX_APPROX = 0, DVL_VMAX_EXACT = 1 };
enum { DVL_WIDTH_EDGE = 0, DVL_WIDTH_VOLUME = 1 };

/* Limits of this build. */
#define DVL_MAX_FIELDS 8          /* M */
#define DVL_MAX_TF_ENTRIES 4096   /* T */
#define DVL_MAX_WIDTH 65536       /* W */
#define DVL_MAX_LEVEL 20          /* logical grid up to 2^20 finest cells */

/* Parameters of one update (paper Eq. 2/3, Sec. 3.2).
 *   P               steepness exponent, >= 0.  When 2P is an integer in
 *                   [0, 16] the widths are bit-exact across CPU and GPU;
 *                   other values use powf (results then agree to a tolerance).
 *   min_importance  minimum importance m >= 0 (paper default 0.025).
 *   width           W, number of pixel bins, 1..DVL_MAX_WIDTH.
 *   min_imp_mode    DVL_MINIMP_BEFORE_SCALE: f = (max(V/maxV, m) 2^L)^P
 *                   DVL_MINIMP_AFTER_POWER:  f = max((V/maxV 2^L)^P, m)
 *   vmax_mode       DVL_VMAX_APPROX: max V from the TF entries the data range
 *                   reaches (Sec. 3.4, Eq. 5/6); DVL_VMAX_EXACT: max over cells.
 *   width_mode      DVL_WIDTH_EDGE: scale 2^L; DVL_WIDTH_VOLUME: 8^L (Sec. 3.1).
 *   want_alpha      1 = also accumulate, per field and pixel, the mean of the
 *                   cells' TF alpha (read with dvl_read_alpha_means; needed by
 *                   dvl_backward); 0 = not (default, slightly faster). */
typedef struct {
    float P;
    float min_importance;
    uint32_t width;
    uint32_t min_imp_mode;
    uint32_t vmax_mode;
    uint32_t width_mode;
    uint32_t want_alpha;
} dvl_params;

/* Destination of dvl_read_bins for one field.  Each pointer may be NULL
 * (skipped); each non-NULL one holds W elements.  mean/min/max are of the
 * normalised field value t in [0, 1] (Sec. 3.3) over the cells covering the
 * pixel; y is the TF alpha of the mean (bar height / polyline y, Sec. 3.3);
 * sum is the float64 sum of t; count is the number of covering cells (the
 * per-pixel counter of Sec. 3.2, shared by all fields).  Empty pixels
 * (count 0) report 0 everywhere. */
typedef struct {
    float* mean;
    float* min;
    float* max;
    float* y;
    double* sum;
    uint32_t* count;
    int mem_kind;
} dvl_bins;

/* Per-update scalars, for checking and display. */
typedef struct {
    float vmax;          /* max V used in Eq. 3 */
    float inv_vmax;      /* float32 reciprocal of vmax (0 if vmax == 0) */
    float f_upper;       /* upper bound of the importance over all cells */
    int32_t Q;           /* fixed-point exponent: width q = rint(f * 2^Q) */
    int32_t i, j;        /* global TF entry range of Eq. 5 */
    int32_t linear;      /* 1 if every width was 0 and equal widths were used */
    int32_t pow_exact;   /* 1 if 2P is an integer in [0, 16] */
    uint64_t F;          /* sum of all fixed-point widths (Eq. 4 total) */
    uint64_t n_cells;
    uint32_t n_fields;
    uint32_t max_level;
    uint32_t entries;    /* 1 if the width pass streamed the cells' kept TF
                            entries (DVL_OPT_ENTRIES), 0 if their field values */
    uint32_t pad;
} dvl_stats;

/* Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * of that device on which all work is issued, or NULL for a library-owned
 * non-blocking stream.  Errors: DVL_ERR_ARG (out NULL), DVL_ERR_CUDA (no such
 * device / no GPU), DVL_ERR_NOMEM. */
int dvl_create(dvl_ctx** out, int device, void* cuda_stream);

/* Waits for the context's work and releases everything it owns.  NULL is a
 * no-op. */
void dvl_destroy(dvl_ctx* ctx);

/* Loads an AMR data set (paper Sec. 2.1: a cell is its lower corner on the
 * logical grid plus its level, 0 = finest, width 2^level).
 *   n_cells   N, 0 <= N < 2^32
 *   lower     3*N int32, structure of arrays: x[0..N), y[0..N), z[0..N);
 *             each cell must satisfy 0 <= lower and lower + 2^level <= 2^20
 *   level     N uint8, <= DVL_MAX_LEVEL
 *   fields    n_fields pointers to N float32 values each (finite)
 * Replaces any previous data set and clears the order and the TFs.
 * Errors: DVL_ERR_ARG, DVL_ERR_RANGE (cell outside the grid, level too high,
 * non-finite value), DVL_ERR_NOMEM, DVL_ERR_CUDA. */
int dvl_load_amr(dvl_ctx* ctx, uint64_t n_cells, const int32_t* lower, const uint8_t* level,
                 uint32_t n_fields, const float* const* fields, int mem_kind);

/* Builds the curve order once per data set (paper Sec. 2.2, Sec. 4): a
 * 63-bit key per cell from its exact centroid 2*lower + 2^level (21 bits per
 * axis), Morton or Hilbert (Skilling's construction), then a stable radix
 * sort of the cells by key; fields and levels are gathered into curve order.
 * Needs LOADED.  Errors: DVL_ERR_ARG (sfc), DVL_ERR_STATE, DVL_ERR_NOMEM,
 * DVL_ERR_TIMEOUT, DVL_ERR_CUDA. */
int dvl_build_order(dvl_ctx* ctx, int sfc);

/* Replaces the field values of the loaded cells (a data change), keeping the
 * cells and their order (re-gathered through the stored permutation).
 * n_fields must equal the loaded count.  Needs ORDERED. */
int dvl_set_fields(dvl_ctx* ctx, uint32_t n_fields, const float* const* fields, int mem_kind);

/* Per-field value scale.  Fields spanning many decades (densities,
 * pressures of astrophysical AMR data) are usually normalised on a log axis:
 * DVL_SCALE_LOG10 replaces the field's values by their log10 before anything
 * else of the update sees them, so the domain normalisation of Sec. 3.3 (and
 * the default TF domain, the field's data range) applies to the log values.
 * A value <= 0 first takes the field's smallest positive value.  The log10
 * is a fixed sequence of correctly rounded float32 operations (argument
 * reduction to [sqrt(2)/2, sqrt(2)), the atanh series, log10(2) split in two
 * floats), within 1.5 ulp of the exact log10, with the same bits on every
 * IEEE float32 implementation of the sequence.  The scale holds until the
 * next dvl_load_amr and is re-applied by dvl_set_fields (a log-scaled field
 * whose new values have no positive value returns to the linear scale, and
 * dvl_set_fields returns DVL_ERR_RANGE after setting the values).  Needs
 * LOADED; once the order is built, the values are re-gathered at once
 * (synchronising) and the value tables are rebuilt by the next update.
 * Errors: DVL_ERR_ARG (field, scale), DVL_ERR_STATE, DVL_ERR_RANGE (log
 * scale for a field without a positive value), DVL_ERR_CUDA. */
enum { DVL_SCALE_LINEAR = 0, DVL_SCALE_LOG10 = 1 };
int dvl_set_field_scale(dvl_ctx* ctx, uint32_t field, int scale);

/* Copies the n_cells values of one field in curve order as the update sees
 * them (after the field's scale).  Host output synchronises; device output
 * is enqueued on the context's stream.  Needs ORDERED.
 * Errors: DVL_ERR_ARG, DVL_ERR_STATE, DVL_ERR_CUDA. */
int dvl_read_values(dvl_ctx* ctx, uint32_t field, float* out, int mem_kind);

/* The data range of every field as the update sees it (after the scales):
 * lo[n_fields], hi[n_fields], host memory.  Synchronising.  Needs LOADED.
 * Errors: DVL_ERR_ARG, DVL_ERR_STATE, DVL_ERR_CUDA. */
int dvl_read_data_range(dvl_ctx* ctx, float* lo, float* hi);

/* Sets the alpha transfer function of one field (paper Sec. 3.3): n_entries
 * alpha values in [0, 1] over the normalised domain, entry a covering
 * t in [a/T, (a+1)/T) (the last entry closed).  The field value v maps to
 * t = clamp((v - domain_lo) / (domain_hi - domain_lo), 0, 1); pass NaN for
 * both bounds to use the field's data range.  All fields must use the same
 * n_entries (2..DVL_MAX_TF_ENTRIES).  `alpha` is host memory; it is copied.
 * Errors: DVL_ERR_ARG (field, size, alpha outside [0,1], lo >= hi),
 * DVL_ERR_STATE (no data loaded). */
int dvl_set_tf(dvl_ctx* ctx, uint32_t field, const float* alpha, uint32_t n_entries,
               float domain_lo, float domain_hi);

/* Sets the alpha transfer functions of all fields in one call, as
 * dvl_set_tf does for each field m with alpha + m*n_entries (field-major,
 * n_fields x n_entries host floats) and the domain (domain[m],
 * domain[n_fields + m]); domain may be NULL for every field's data range.
 * n_fields must equal the data set's field count.  Every argument is checked
 * before any table changes, so a refused call leaves the tables as they were.
 * Errors: DVL_ERR_ARG, DVL_ERR_STATE (no data loaded). */
int dvl_set_tfs(dvl_ctx* ctx, uint32_t n_fields, const float* alpha, uint32_t n_entries, const float* domain);

/* Enqueues one DVL update (paper Sec. 3-4): per cell and field the TF alpha,
 * the local variation V (Eq. 1), the importance (Eq. 3), a fixed-point width,
 * the device-wide prefix sum (Eq. 4), the projection of every cell into the
 * pixels its span touches with per-pixel sum/min/max/count (Sec. 3.2), and
 * the per-pixel mean and alpha.  Asynchronous; read results with
 * dvl_read_bins.  The first update after a TF-domain, table-size or data
 * change also rebuilds the context's value tables and (DVL_OPT_ENTRIES, at
 * most 256 table entries) the per-cell TF entries, n_fields + 1 bytes a
 * cell (the entries and a copy of the levels in their order) held until the
 * data set is replaced; later alpha-only edits stream those bytes instead of
 * the field values.
 * Errors: DVL_ERR_ARG (params), DVL_ERR_STATE, DVL_ERR_NOMEM,
 * DVL_ERR_CUDA.  Device-side failures (DVL_ERR_RANGE for a width bound that
 * cannot be represented, DVL_ERR_TIMEOUT) surface at the next synchronising
 * call. */
int dvl_update(dvl_ctx* ctx, const dvl_params* params);

/* Sets every field's alpha table from K control points per field
 * (differentiable parameterisation; not in the paper, whose TFs are edited
 * directly): control point k sits at k/(K-1), table entry e at e/(T-1) is the
 * linear interpolation of its two neighbouring control points, evaluated in
 * float32 as x = e(K-1)/(T-1), k0 = floor(x) (at most K-2), w = x - k0,
 * A = c[k0] + w (c[k0+1] - c[k0]).
 *   ctrl     M x K floats in [0, 1] (field-major), host or device per mem_kind
 *   K        2..1024 control points; T: 2..DVL_MAX_TF_ENTRIES entries
 *   domain   2*M floats lo[M], hi[M] (host; NaN/NaN = data range) or NULL
 *            for the data range of every field
 * The tables stay on the device (no host round trip).  Errors: DVL_ERR_ARG,
 * DVL_ERR_STATE (no data loaded); control points outside [0, 1] in device
 * memory are reported as DVL_ERR_RANGE by the next synchronising call. */
int dvl_set_tf_ctrl(dvl_ctx* ctx, const float* ctrl, uint32_t K, uint32_t T, const float* domain,
                    int mem_kind);

/* Per-pixel mean of the cells' TF alpha of the last update (which must have
 * had want_alpha = 1): abar[m][p] = (1/count_p) sum over the cells covering
 * pixel p of A_m[entry_m(cell)] -- the differentiable counterpart of the bin
 * mean (the mean of the normalised value has zero gradient with respect to the
 * TF).  out: M x W floats (field-major), host or device.  Synchronises for a
 * host destination; a device copy is ordered on the context's stream. */
int dvl_read_alpha_means(dvl_ctx* ctx, float* out, int mem_kind);

/* Adjoint of dvl_read_alpha_means with the cell-to-pixel assignment and the
 * cells' TF entries held fixed at the last update: given g[m][p] = dL/dabar,
 * returns dL/dctrl[m][k] = sum_e (sum over (cell, pixel) pairs with entry e of
 * g[m][p] / count_p) * dA_m[e]/dctrl[m][k] (the interpolation weights of
 * dvl_set_tf_ctrl, in float64).  Needs an update with want_alpha = 1 after
 * dvl_set_tf_ctrl.
 *   grad_abar   M x W floats, memory kind mem_in
 *   grad_ctrl   M x K floats (output), memory kind mem_out
 * Synchronises unless both buffers are device memory (then the work is
 * ordered on the context's stream and device-side errors surface at the next
 * synchronising call).  Errors: DVL_ERR_ARG, DVL_ERR_STATE. */
int dvl_backward(dvl_ctx* ctx, const float* grad_abar, int mem_in, float* grad_ctrl, int mem_out);

/* Copies the bins of one field of the last update into `out` (see dvl_bins).
 * Synchronises the context's stream for host destinations; device
 * destinations are copied on the stream and the call then synchronises too,
 * so device-side errors of the update are reported here. */
int dvl_read_bins(dvl_ctx* ctx, uint32_t field, const dvl_bins* out);

/* The bins of every field of the last update in one call: mean, min, max, y
 * and sum hold n_fields*W elements, field m's row starting at element m*W
 * (the layout dvl_read_bins fills one row of); count holds W (shared by the
 * fields).  NULL members are skipped.  One copy per array and one
 * synchronisation of the context's stream, whatever the number of fields;
 * device-side errors of the update are reported here (the buffers' contents
 * are then unspecified).  Errors: DVL_ERR_ARG,
 * DVL_ERR_STATE, DVL_ERR_CUDA, and the device-side DVL_ERR_TIMEOUT and
 * DVL_ERR_RANGE. */
int dvl_read_bins_all(dvl_ctx* ctx, const dvl_bins* out);

/* Scalars of the last update (synchronises). */
int dvl_get_stats(dvl_ctx* ctx, dvl_stats* out);

/* Copies the sorted curve keys (keys[k] = key of the k-th cell in curve
 * order, N u64) and the permutation (perm[k] = input index of the k-th cell
 * in curve order, N u32).  Either pointer may be NULL.  Needs ORDERED;
 * synchronises. */
int dvl_read_order(dvl_ctx* ctx, uint64_t* keys, uint32_t* perm, int mem_kind);

/* Copies the fixed-point width q of every cell of the last update, in curve
 * order (N u64).  A checking aid: recomputes the widths with the update's
 * constants.  Synchronises. */
int dvl_read_widths(dvl_ctx* ctx, uint64_t* q, int mem_kind);

/* Waits for all enqueued work; returns the first device-side error
 * (DVL_ERR_TIMEOUT, DVL_ERR_RANGE) raised since the last synchronising call. */
int dvl_sync(dvl_ctx* ctx);

/* Average device time per stage, in milliseconds, over the dvl_update calls
 * made with DVL_OPT_TIMING = 1 since the previous dvl_get_timings (CUDA events
 * recorded on the context's stream between the kernels).  ms[0] = constants
 * and clearing (plus the exact max-V pass if selected), ms[1] = width pass
 * with the prefix scan, ms[2] = placement/reduction pass, ms[3] = finalize;
 * if n >= 5, ms[4] = number of updates averaged.  n >= 4.  Synchronises and
 * resets the collection.  DVL_ERR_STATE if no timed update is pending. */
int dvl_get_timings(dvl_ctx* ctx, double* ms, int n);

/* Tuning and fault-injection options (for tests).
 *   DVL_OPT_SPIN_LIMIT      iteration limit of every device-side wait
 *                           (default 1<<22; each iteration sleeps ~100 ns)
 *   DVL_OPT_FAULT_NO_PUBLISH  1 = in the next update's width pass, a bounded
 *                           device-side wait is made to run out (tests
 *                           DVL_ERR_TIMEOUT): the first warp waits on a signal
 *                           that nothing sends or, where that pass reads the
 *                           cells directly (rows not 16-byte aligned), the
 *                           first tile of its look-back scan never publishes
 *                           its sum; reset after one update.
 *   DVL_OPT_TIMING          1 = record per-stage CUDA events in every
 *                           dvl_update (read with dvl_get_timings); 0 = off
 *                           (default).  A timed dvl_update_batch runs its
 *                           kernels as plain launches instead of the graph
 *                           (stages: prepare, pass A, bins, -).
 *   DVL_OPT_ENTRIES         1 (default) = with alpha tables of at most 256
 *                           entries, dvl_update keeps each cell's TF entry per
 *                           field and a copy of its level (n_fields + 1 bytes
 *                           a cell, built in the first update after a
 *                           TF-domain, table-size or data change, like the
 *                           value tables) and its width pass reads those
 *                           instead of the field values; 0 = the
 *                           width pass reads the field values.  The results
 *                           are the same bit for bit. */
enum { DVL_OPT_SPIN_LIMIT = 1, DVL_OPT_FAULT_NO_PUBLISH = 2, DVL_OPT_TIMING = 3, DVL_OPT_ENTRIES = 4 };
int dvl_set_option(dvl_ctx* ctx, int option, int64_t value);

/* Line-plot image of the bins of the last dvl_update (the RasterizeLines
 * step after the update, Sec. 4, Fig. 1), headless: an height x W image, row 0
 * at the top, column p = bin p, row-major bytes.
 *   value_kind  DVL_PLOT_MEAN (mean of the normalised values) or DVL_PLOT_Y
 *               (alpha of the mean, the bar heights of Fig. 1)
 *   lines       bit m set where field m's polyline covers the pixel: a bin
 *               value v maps to row r = clamp(floor((1 - v)(height - 1) +
 *               1/2), 0, height - 1) (float32 steps), and column p covers
 *               the rows between r_p, r_p - trunc((r_p - r_{p-1})/2) and
 *               r_p + trunc((r_{p+1} - r_p)/2)
 *   bars        1 from r_p of field bar_field down to the last row, else 0
 * Either output may be NULL; host or device memory per mem_kind (host: the
 * call synchronises).  height in [1, 65536].  Errors: DVL_ERR_ARG,
 * DVL_ERR_STATE (no update has run), DVL_ERR_NOMEM, DVL_ERR_CUDA. */
enum { DVL_PLOT_MEAN = 0, DVL_PLOT_Y = 1 };
int dvl_rasterize(dvl_ctx* ctx, uint32_t height, uint32_t value_kind, uint32_t bar_field, uint8_t* lines,
                  uint8_t* bars, int mem_kind);

/* Brushing and linking (Sec. 3.5).  A pixel ROI [p0, p1] (inclusive, < W) of
 * the last dvl_update's plot selects the cells whose span touches one of its
 * pixels: one run [first, last] of the curve order (n_cells = 0 when empty),
 * with its first and last curve keys, the compact ROI the 3D view tests cells
 * against.  mask (optional, n_cells bytes, host or device per mem_kind):
 * 1 for the selected cells, 0 otherwise, in the order the cells were loaded.
 * Needs the last update to have run with want_alpha = 0 (DVL_ERR_STATE
 * otherwise).  Synchronises the stream. */
typedef struct dvl_roi {
    uint64_t first, last, n_cells;        /* curve-order indices, inclusive */
    uint64_t key_first, key_last;         /* their curve keys */
} dvl_roi;
int dvl_brush(dvl_ctx* ctx, uint32_t p0, uint32_t p1, dvl_roi* out, uint8_t* mask, int mem_kind);

/* The linked selection in the 3D view: mask[c] = 1 (input order) when cell
 * c's curve key lies in one of R inclusive key ranges (host array ranges[2r],
 * ranges[2r+1]; R <= DVL_MAX_SELECT_RANGES).  mask holds n_cells bytes, host
 * or device per mem_kind. */
enum { DVL_MAX_SELECT_RANGES = 1024 };
int dvl_select_keys(dvl_ctx* ctx, const uint64_t* ranges, uint32_t R, uint8_t* mask, int mem_kind);

/* Batched update: K transfer functions, each with any number of viewport
 * widths, over the loaded data set (paper Sec. 3.3-3.4 per (TF, width) pair;
 * the batching itself is not in the paper -- it serves many clients editing
 * TFs of one resident data set).  Results equal dvl_update's for the same TF,
 * domain, params and width, bit for bit.
 *   alphas      K x n_fields x n_entries alpha tables in [0, 1], TF-major
 *               (TF k, field m at alphas + (k*n_fields + m)*n_entries);
 *               host or device per mem_kind
 *   domain      host, 2*n_fields floats (lo[0..M), hi[0..M)), shared by all K
 *               TFs; NaN/NaN = the field's data range; NULL = all data ranges
 *   params      P, min_importance, min_imp_mode, width_mode as dvl_update;
 *               vmax_mode must be DVL_VMAX_APPROX, want_alpha 0; width ignored
 *   pair_tf     host, n_pairs TF indices (< K)
 *   pair_width  host, n_pairs widths in [1, DVL_MAX_WIDTH]
 * K <= DVL_MAX_BATCH_TF, 1 <= n_pairs <= DVL_MAX_BATCH_PAIRS.  The first call
 * with a new shape (n_fields, n_entries, K, P == 1, the pair list) times a few
 * launch configurations and keeps the fastest; later calls of that shape
 * replay one captured CUDA graph.  Asynchronous on the context's stream.
 * Errors: DVL_ERR_ARG, DVL_ERR_STATE (no order built), DVL_ERR_NOMEM,
 * DVL_ERR_CUDA; device-side errors (DVL_ERR_TIMEOUT, DVL_ERR_RANGE) surface in
 * dvl_read_batch_bins. */
enum { DVL_MAX_BATCH_TF = 256, DVL_MAX_BATCH_PAIRS = 4096 };
int dvl_update_batch(dvl_ctx* ctx, const float* alphas, uint32_t K, uint32_t n_entries, int mem_kind,
                     const float* domain, const dvl_params* params, const uint32_t* pair_tf,
                     const uint32_t* pair_width, uint32_t n_pairs);

/* Bins of pair `pair` of the last dvl_update_batch (layout as dvl_read_bins
 * with W = pair_width[pair]).  Synchronises the stream. */
int dvl_read_batch_bins(dvl_ctx* ctx, uint32_t pair, uint32_t field, const dvl_bins* out);

/* All bins of the last dvl_update_batch in one copy per array: pair q's
 * field m starts at element bin_off(q) + m*W_q of mean/min/max/y/sum and its
 * counts at cnt_off(q) of count, where bin_off(q) = sum over earlier pairs of
 * n_fields*W and cnt_off(q) = sum over earlier pairs of W.  Buffers must hold
 * the totals.  Synchronises the stream. */
int dvl_read_batch_all(dvl_ctx* ctx, const dvl_bins* out);

/* As dvl_read_batch_all, but only queues the copies on the context's stream
 * and returns (no synchronisation, no device-error check): host buffers must
 * be pinned and stay valid until the stream has passed the copies
 * (dvl_sync, or an event / host callback on dvl_stream). */
int dvl_read_batch_all_async(dvl_ctx* ctx, const dvl_bins* out);

/* The CUDA stream (cudaStream_t) the context runs its work on. */
void* dvl_stream(dvl_ctx* ctx);

/* Launch configuration the batch autotuner chose for the last batch shape:
 * out[0] = TFs per shared-memory group, out[1] = pass-A CTAs per SM,
 * out[2] = 1 if the last call replayed a captured graph. */
int dvl_batch_config(dvl_ctx* ctx, int32_t out[3]);

/* One DVL update that allocates no device memory, for callers that must not
 * call cudaMalloc or cudaFree at that point (a render or UI callback inside a
 * memory budget owned by someone else, a process limited to a fixed pool, code
 * that must not cause the device-wide synchronisation cudaFree implies).  The
 * paper has no counterpart: it is an interface variant of dvl_update.
 *
 * Inputs and outputs are the caller's device buffers; no context is used.  The
 * working memory beyond them lives in one fixed 4 MiB array inside the library
 * that every GPU loading the library keeps until the process exits; this caps
 * n_cells at 476,749,824 (larger counts return DVL_ERR_RANGE before any GPU
 * work).  The first call on a device looks up that array's device address
 * (with the device current) and keeps it for the life of the process; make
 * that first call before any stream capture.  A cudaDeviceReset destroys the
 * array's memory with the context, so the kept address is then stale: do not
 * use this entry point on a device after resetting it.
 * All calls share the array and it keeps the previous call's contents (each
 * call re-initialises what must start fresh), so calls that overlap on the GPU
 * -- on different streams or host threads -- race and must be serialised by
 * the caller.
 *   cuda_stream  stream of the current device the work runs on (NULL = legacy
 *                default stream); the call waits for that stream to finish
 *                its work before returning (it reads back an error word)
 *   fields       device, cells in curve order, field m at fields + m*pitch;
 *                16-byte aligned, pitch a multiple of 4 and >= n_cells rounded
 *                up to a multiple of 4 (the buffer must hold n_fields*pitch
 *                floats; values finite)
 *   level        device, n_cells levels rounded up to a multiple of 4 bytes,
 *                4-byte aligned
 *   alpha        device, n_fields x n_entries alpha tables in [0, 1]
 *   domain       host, 2*n_fields floats: lo[0..M), hi[0..M); NaN/NaN = data
 *                range (as dvl_set_tf)
 *   params       as dvl_update (want_alpha must be 0)
 *   out          device buffers of n_fields*W (mean, min, max, y, sum) and W
 *                (count) elements, field-major; all six required,
 *                mem_kind = DVL_MEM_DEVICE
 * Results, for the same cells in the same order, against dvl_update's:
 * counts, min and max bit-identical; sums and means within 1e-5 relative
 * (this call places the cells with a second pass over them instead of
 * dvl_update's prefix tables, so sums are added in another order); y the
 * same except where a mean lies that close to a TF bucket boundary.  Errors:
 * DVL_ERR_ARG, DVL_ERR_RANGE (size cap, non-finite value, width bound),
 * DVL_ERR_TIMEOUT, DVL_ERR_CUDA. */
int dvl_update_noalloc(void* cuda_stream, uint64_t n_cells, uint32_t n_fields, const float* fields,
                       size_t pitch, const uint8_t* level, uint32_t n_entries, const float* alpha,
                       const float* domain, const dvl_params* params, const dvl_bins* out);

/* Static message for a status code. */
const char* dvl_status_string(int status);

/* Message of the last failing call on ctx (empty if none); never NULL. */
const char* dvl_last_error(dvl_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DVL_H */
