/*
 * CPU oracle for the DVL computation -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain sequential restatement of the paper's method (Sec. 2.1, 2.2, 3.1-3.4),
 * written for a reader checking it against the equations, not for speed.  Only
 * the tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * CUDA library shares no code with it.  Build: gcc -O2 -ffp-contract=off
 * (no fused multiply-add, no fast-math) so that every float operation below is
 * one correctly rounded IEEE operation.
 *
 * Readings of points the paper leaves open are stated where they are used.
 * orc_update_mt and orc_keys_mt spread the same per-cell arithmetic over host
 * threads (OpenMP) for the all-cores CPU baseline and for oracle runs at
 * benchmark sizes; their results equal the sequential functions' bit for bit.
 */
#include "dvl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define SFC_BITS 21              /* bits per axis of the centroid grid */
#define MAX_LEVEL 20             /* logical grid up to 2^20 finest cells */

/* ------------------------------------------------------------------------- */
/* Space-filling-curve keys (Sec. 2.2; cell = lower corner + level, Sec. 2.1) */
/* ------------------------------------------------------------------------- */

/* Morton (Z-order) code: bit k of axis d becomes key bit 3k+d (x lowest). */
static uint64_t morton3(const uint32_t c[3])
{
    uint64_t key = 0;
    for (int k = 0; k < SFC_BITS; ++k)
        for (int d = 0; d < 3; ++d)
            key |= (uint64_t)((c[d] >> k) & 1u) << (3 * k + d);
    return key;
}

/* Hilbert code after J. Skilling, "Programming the Hilbert curve", AIP Conf.
 * Proc. 707 (2004): the axes are turned into the "transposed" Hilbert index
 * by undoing, from the coarsest bit plane to the finest, the reflections and
 * axis exchanges the curve applies below each plane, then Gray-coding across
 * the axes; the transposed index is read out one bit plane at a time, axis 0
 * first.  The number of bit planes is fixed (21) so the key of a cell does
 * not depend on the extent of the data set. */
static uint64_t hilbert3(const uint32_t c[3])
{
    uint32_t X[3] = {c[0], c[1], c[2]};
    const uint32_t top = 1u << (SFC_BITS - 1);
    for (uint32_t plane = top; plane > 1; plane >>= 1) {
        uint32_t below = plane - 1;
        for (int d = 0; d < 3; ++d) {
            if (X[d] & plane) {
                X[0] ^= below;                      /* reflect the lower bits of axis 0 */
            } else {
                uint32_t diff = (X[0] ^ X[d]) & below;  /* swap lower bits of axes 0 and d */
                X[0] ^= diff;
                X[d] ^= diff;
            }
        }
    }
    X[1] ^= X[0];                                   /* Gray code across axes */
    X[2] ^= X[1];
    uint32_t flip = 0;
    for (uint32_t plane = top; plane > 1; plane >>= 1)
        if (X[2] & plane) flip ^= plane - 1;
    for (int d = 0; d < 3; ++d) X[d] ^= flip;
    uint64_t key = 0;
    for (int b = SFC_BITS - 1; b >= 0; --b)
        for (int d = 0; d < 3; ++d) key = (key << 1) | ((X[d] >> b) & 1u);
    return key;
}

int orc_keys(uint64_t n, const int32_t* lx, const int32_t* ly, const int32_t* lz,
             const uint8_t* level, int sfc, uint64_t* keys)
{
    if (sfc != ORC_SFC_MORTON && sfc != ORC_SFC_HILBERT) return -1;
    for (uint64_t i = 0; i < n; ++i) {
        int32_t lo[3] = {lx[i], ly[i], lz[i]};
        if (level[i] > MAX_LEVEL) return -5;
        int64_t w = (int64_t)1 << level[i];
        uint32_t c[3];
        for (int d = 0; d < 3; ++d) {
            if (lo[d] < 0 || (int64_t)lo[d] + w > ((int64_t)1 << MAX_LEVEL)) return -5;
            c[d] = (uint32_t)(2 * (int64_t)lo[d] + w);  /* centroid, half-cell units */
        }
        keys[i] = sfc == ORC_SFC_MORTON ? morton3(c) : hilbert3(c);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Stable order by key (Sec. 4: computed once, never changes)                */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t key; uint32_t idx; } kv;

static int kv_cmp(const void* a, const void* b)
{
    const kv* x = (const kv*)a;
    const kv* y = (const kv*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);   /* ties keep input order */
}

int orc_order(uint64_t n, const uint64_t* keys, uint32_t* perm)
{
    if (n > 0xFFFFFFFFull) return -1;
    kv* a = (kv*)malloc(sizeof(kv) * (n ? n : 1));
    if (!a) return -3;
    for (uint64_t i = 0; i < n; ++i) { a[i].key = keys[i]; a[i].idx = (uint32_t)i; }
    qsort(a, n, sizeof(kv), kv_cmp);
    for (uint64_t i = 0; i < n; ++i) perm[i] = a[i].idx;
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Per-update setup: normalisation, Eq. 5 ranges, Eq. 6 approximation         */
/* ------------------------------------------------------------------------- */

/* Normalised field value t = clamp((v - lo) * s, 0, 1) with s the float32
 * reciprocal of (hi - lo) (Sec. 3.3: the field intensity is normalised before
 * the transfer-function lookup).  s = 0 for an empty or non-finite span. */
static float norm_scale(float lo, float hi)
{
    float span = hi - lo;
    if (!(span > 0.0f) || !isfinite(span)) return 0.0f;
    return 1.0f / span;
}

static float normalise(float v, float lo, float s)
{
    float t = (v - lo) * s;
    if (!(t > 0.0f)) t = 0.0f;                  /* also maps NaN to 0 */
    if (t > 1.0f) t = 1.0f;
    return t;
}

/* Transfer-function entry of a normalised value: nearest-lower bucket of T
 * equal buckets over [0, 1], the last bucket closed. */
static uint32_t tf_entry(float t, uint32_t T)
{
    float x = t * (float)T;
    uint32_t a = (uint32_t)floorf(x);
    return a > T - 1 ? T - 1 : a;
}

/* x^P for the steepness exponent of Eq. 2/3.  When 2P is an integer in
 * [0, 16] the power is a fixed sequence of correctly rounded operations
 * (square root once if 2P is odd, then left-to-right products); 0^0 = 1.
 * Otherwise powf is used and results are compared with a tolerance. */
static int pow_is_exact(float P)
{
    float n2 = 2.0f * P;
    return n2 >= 0.0f && n2 <= 16.0f && floorf(n2) == n2;
}

static float pow_steep(float x, float P)
{
    if (!pow_is_exact(P)) return powf(x, P);
    int n2 = (int)(2.0f * P);
    if (n2 == 0) return 1.0f;
    float b;
    int k;
    if (n2 & 1) { b = sqrtf(x); k = n2; } else { b = x; k = n2 / 2; }
    float y = b;
    for (int i = 1; i < k; ++i) y = y * b;
    return y;
}

static float pow2f_int(int e) { return ldexpf(1.0f, e); }

/* Importance of one cell, Eq. 3, with the minimum importance of Eq. 2.
 *   r = V * (1/maxV)            (float32 reciprocal of max V, Sec. 3.4)
 *   before-scale mode:  f = (max(r, m) * 2^L)^P
 *   after-power  mode:  f = max((r * 2^L)^P, m)
 * The cell-width factor is 2^L (edge) or 8^L (volume, the alternative the
 * paper mentions in Sec. 3.1). */
static float importance(float V, float inv_vmax, int level, const orc_params* p)
{
    float r = V * inv_vmax;
    int e = (int)level * (p->width_mode == ORC_WIDTH_VOLUME ? 3 : 1);
    float f;
    if (p->min_imp_mode == ORC_MINIMP_BEFORE_SCALE) {
        if (r < p->min_importance) r = p->min_importance;
        f = pow_steep(r * pow2f_int(e), p->P);
    } else {
        f = pow_steep(r * pow2f_int(e), p->P);
        if (f < p->min_importance) f = p->min_importance;
    }
    return f;
}

static int bitlen64(uint64_t x)
{
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

/* ------------------------------------------------------------------------- */
/* One DVL update                                                            */
/* ------------------------------------------------------------------------- */

/* Fixed-point widths.  Every width is f <= f_upper (each operation of Eq. 3 is
 * monotone for non-negative arguments and V <= 1), so with f_upper <= 2^e the
 * widths q = rint(f * 2^Q) are at most 2^(Q+e).  Q + e is capped at 31 (every
 * width fits in 32 bits) and at 62 - nb for n < 2^nb cells (the total stays
 * below 2^62): the prefix sum of Eq. 4 is then exact integer arithmetic and
 * does not depend on summation order.  Returns -5 when not representable. */
static int fixed_point(float Vmax, float inv_vmax, int max_level, uint64_t n, const orc_params* prm,
                       float* f_upper_out, int* Q_out)
{
    float f_upper = importance(1.0f, inv_vmax, max_level, prm);
    if (Vmax == 0.0f) f_upper = importance(0.0f, 0.0f, max_level, prm);
    if (!isfinite(f_upper)) return -5;
    int ex = 0;
    frexpf(f_upper, &ex);                     /* f_upper <= 2^ex */
    if (!pow_is_exact(prm->P)) ex += 1;       /* powf is not monotone to the ulp */
    int cap = 62 - bitlen64(n);
    if (cap > 31) cap = 31;
    int Q = cap - ex;
    if (Q > 120) Q = 120;
    if (Q < -120) return -5;
    *f_upper_out = f_upper;
    *Q_out = Q;
    return 0;
}

int orc_update(uint64_t n, uint32_t M, const float* fields, const uint8_t* level,
               uint32_t T, const float* alpha, const float* dom_lo, const float* dom_hi,
               const orc_params* prm, double* sum, float* vmin, float* vmax, float* mean,
               double* mean64, float* y, uint32_t* count, uint64_t* q_out, uint32_t* b1_out,
               uint32_t* b2_out, orc_stats* st)
{
    const uint32_t W = prm->width;
    if (M < 1 || M > 16 || T < 2 || W < 1 || !sum || !vmin || !vmax || !count) return -1;
    for (uint64_t e = 0; e < (uint64_t)M * T; ++e)
        if (!(alpha[e] >= 0.0f && alpha[e] <= 1.0f)) return -1;

    /* Transfer-function domain per field: given, or the data range. */
    float lo[16], s[16], dmin[16], dmax[16];
    for (uint32_t m = 0; m < M; ++m) {
        const float* v = fields + (uint64_t)m * n;
        float a = INFINITY, b = -INFINITY;
        for (uint64_t c = 0; c < n; ++c) {
            if (v[c] < a) a = v[c];
            if (v[c] > b) b = v[c];
        }
        if (n == 0) { a = 0.0f; b = 0.0f; }
        dmin[m] = a;
        dmax[m] = b;
        float l = dom_lo[m], h = dom_hi[m];
        if (isnan(l) && isnan(h)) { l = a; h = b; }
        lo[m] = l;
        s[m] = norm_scale(l, h);
    }

    /* Max local variation.  Approximate mode, Sec. 3.4: the TF entries the
     * data reaches are [i_m, j_m] per field (entries of the data minimum and
     * maximum); Eq. 5 takes their union [i, j]; Eq. 6 takes the largest
     * spread max_m A(m,a) - min_m A(m,a) over a in [i, j].  Entries are
     * paired across fields by index, exactly as Eq. 6 is written. */
    int gi = (int)T - 1, gj = 0;
    for (uint32_t m = 0; m < M; ++m) {
        int im = (int)tf_entry(normalise(dmin[m], lo[m], s[m]), T);
        int jm = (int)tf_entry(normalise(dmax[m], lo[m], s[m]), T);
        if (im < gi) gi = im;
        if (jm > gj) gj = jm;
    }
    if (gi > gj) { gi = 0; gj = 0; }
    float Vmax = 0.0f;
    if (prm->vmax_mode == ORC_VMAX_APPROX) {
        for (int a = gi; a <= gj; ++a) {
            float hi = alpha[a], lw = alpha[a];
            for (uint32_t m = 1; m < M; ++m) {
                float x = alpha[(uint64_t)m * T + a];
                if (x > hi) hi = x;
                if (x < lw) lw = x;
            }
            if (hi - lw > Vmax) Vmax = hi - lw;
        }
    } else {
        /* Exact mode: max over cells of Eq. 1 (the reduction Sec. 3.4 avoids). */
        for (uint64_t c = 0; c < n; ++c) {
            float hi = 0.0f, lw = 1.0f;
            for (uint32_t m = 0; m < M; ++m) {
                float al = alpha[(uint64_t)m * T + tf_entry(normalise(fields[(uint64_t)m * n + c], lo[m], s[m]), T)];
                if (al > hi) hi = al;
                if (al < lw) lw = al;
            }
            if (hi - lw > Vmax) Vmax = hi - lw;
        }
    }
    float inv_vmax = Vmax > 0.0f ? 1.0f / Vmax : 0.0f;

    int max_level = 0;
    for (uint64_t c = 0; c < n; ++c)
        if (level[c] > max_level) max_level = level[c];
    float f_upper = 0.0f;
    int Q = 0;
    if (fixed_point(Vmax, inv_vmax, max_level, n, prm, &f_upper, &Q)) return -5;
    float scale = pow2f_int(Q);

    uint64_t* q = q_out ? q_out : (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    if (!q) return -3;
    u128 F = 0;
    for (uint64_t c = 0; c < n; ++c) {
        /* Eq. 1: local variation of the per-field alpha (the intensities
         * I(m,h) come from the alpha transfer function, Sec. 3). */
        float hi = 0.0f, lw = 1.0f;
        for (uint32_t m = 0; m < M; ++m) {
            float t = normalise(fields[(uint64_t)m * n + c], lo[m], s[m]);
            float al = alpha[(uint64_t)m * T + tf_entry(t, T)];
            if (al > hi) hi = al;
            if (al < lw) lw = al;
        }
        float V = hi - lw;
        float f = importance(V, inv_vmax, level[c], prm);   /* Eq. 3 */
        q[c] = (uint64_t)nearbyintf(f * scale);              /* round half to even */
        F += q[c];
    }
    int linear = 0;
    if (F == 0 && n > 0) {             /* all widths 0: fall back to equal widths */
        linear = 1;
        for (uint64_t c = 0; c < n; ++c) q[c] = 1;
        F = n;
    }

    /* Bins (Sec. 3.2): cell c spans [E_c, I_c) with E_c = F(c-1), I_c = F(c)
     * (Eq. 4), i.e. x in [E_c/F * W, I_c/F * W).  Pixel k covers
     * [k, k+1) of that axis; the cell adds its value to every pixel its span
     * touches: b1 = floor(E W / F), b2 = ceil(I W / F) - 1 (a zero-width cell
     * touches only b1), clamped to W-1.  The cell's value is its normalised
     * field value t; the per-pixel counter is shared by all fields. */
    for (uint64_t k = 0; k < (uint64_t)M * W; ++k) { sum[k] = 0.0; vmin[k] = INFINITY; vmax[k] = -INFINITY; }
    for (uint32_t k = 0; k < W; ++k) count[k] = 0;
    u128 E = 0;
    for (uint64_t c = 0; c < n; ++c) {
        u128 I = E + q[c];
        u128 b1 = E * W / F;
        u128 b2 = I > E ? (I * W + F - 1) / F - 1 : b1;
        if (b1 > W - 1) b1 = W - 1;
        if (b2 > W - 1) b2 = W - 1;
        if (b1_out) b1_out[c] = (uint32_t)b1;
        if (b2_out) b2_out[c] = (uint32_t)b2;
        for (uint32_t p = (uint32_t)b1; p <= (uint32_t)b2; ++p) {
            count[p] += 1;
            for (uint32_t m = 0; m < M; ++m) {
                float t = normalise(fields[(uint64_t)m * n + c], lo[m], s[m]);
                uint64_t k = (uint64_t)m * W + p;
                sum[k] += (double)t;
                if (t < vmin[k]) vmin[k] = t;
                if (t > vmax[k]) vmax[k] = t;
            }
        }
        E = I;
    }

    /* ApplyWeights and ApplyTransFunc (Sec. 3.2, 3.3, 4): mean per pixel, then
     * the alpha of the mean is the bar height / polyline y.  Empty pixels
     * (none exist when F > 0) report 0. */
    for (uint32_t m = 0; m < M; ++m)
        for (uint32_t p = 0; p < W; ++p) {
            uint64_t k = (uint64_t)m * W + p;
            double mu = count[p] ? sum[k] / (double)count[p] : 0.0;
            float mf = (float)mu;
            if (mean64) mean64[k] = mu;
            if (mean) mean[k] = mf;
            if (y) y[k] = count[p] ? alpha[(uint64_t)m * T + tf_entry(mf, T)] : 0.0f;
            if (!count[p]) { vmin[k] = 0.0f; vmax[k] = 0.0f; }
        }

    if (st) {
        st->vmax = Vmax;
        st->inv_vmax = inv_vmax;
        st->f_upper = f_upper;
        st->Q = Q;
        st->i = gi;
        st->j = gj;
        st->linear = linear;
        st->pow_exact = pow_is_exact(prm->P);
        st->F = (uint64_t)F;
    }
    if (!q_out) free(q);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The same update spread over host threads (OpenMP)                         */
/* ------------------------------------------------------------------------- */

/* Contiguous share [*b, *e) of n items for thread t of nt. */
static void share(uint64_t n, int nt, int t, uint64_t* b, uint64_t* e)
{
    *b = n / (uint64_t)nt * (uint64_t)t + (n % (uint64_t)nt < (uint64_t)t ? n % (uint64_t)nt : (uint64_t)t);
    *e = *b + n / (uint64_t)nt + ((uint64_t)t < n % (uint64_t)nt ? 1 : 0);
}

/* orc_keys over n_threads contiguous ranges of the cells at once; every key
 * is orc_keys' own, so the output is identical. */
int orc_keys_mt(uint64_t n, const int32_t* lx, const int32_t* ly, const int32_t* lz,
                const uint8_t* level, int sfc, uint64_t* keys, int n_threads)
{
    if (n_threads < 1) return -1;
    int rc = 0;
#pragma omp parallel for num_threads(n_threads) schedule(static, 1) reduction(min : rc)
    for (int t = 0; t < n_threads; ++t) {
        uint64_t b, e;
        share(n, n_threads, t, &b, &e);
        int r = orc_keys(e - b, lx + b, ly + b, lz + b, level + b, sfc, keys + b);
        if (r < rc) rc = r;
    }
    return rc;
}

/* orc_update's result, bit for bit, computed by n_threads threads.  Only the
 * distribution of the work differs:
 *  - per-field data range and deepest level: each thread scans one contiguous
 *    range of cells; the partial results are combined in range order with the
 *    same comparisons, so the first occurrence of an extreme wins as in the
 *    sequential scan;
 *  - widths (Eq. 1, 3 and the fixed point): independent per cell; F is an
 *    exact integer sum, independent of order;
 *  - prefix of Eq. 4: per-range integer totals, their exclusive prefix in
 *    range order, then each range's cells in order (exact integers);
 *  - bins: each thread owns a contiguous run of pixels and visits, in curve
 *    order, the cells whose span touches them, so every pixel receives its
 *    cells' values in the same order as in orc_update (b1 and b2 are
 *    non-decreasing in curve order, so those cells are one run).
 * Setup steps of O(M T) work are the same code as in orc_update. */
int orc_update_mt(uint64_t n, uint32_t M, const float* fields, const uint8_t* level,
                  uint32_t T, const float* alpha, const float* dom_lo, const float* dom_hi,
                  const orc_params* prm, double* sum, float* vmin, float* vmax, float* mean,
                  double* mean64, float* y, uint32_t* count, uint64_t* q_out, uint32_t* b1_out,
                  uint32_t* b2_out, orc_stats* st, int n_threads)
{
    const uint32_t W = prm->width;
    const int nt = n_threads;
    if (nt < 1 || nt > 4096) return -1;
    if (M < 1 || M > 16 || T < 2 || W < 1 || !sum || !vmin || !vmax || !count) return -1;
    for (uint64_t e = 0; e < (uint64_t)M * T; ++e)
        if (!(alpha[e] >= 0.0f && alpha[e] <= 1.0f)) return -1;

    /* data range per field: per-range first extremes, combined in range order */
    float* part = (float*)malloc(sizeof(float) * 2 * 16 * (size_t)nt);
    int* plev = (int*)malloc(sizeof(int) * (size_t)nt);
    if (!part || !plev) { free(part); free(plev); return -3; }
#pragma omp parallel for num_threads(nt) schedule(static, 1)
    for (int t = 0; t < nt; ++t) {
        uint64_t b, e;
        share(n, nt, t, &b, &e);
        for (uint32_t m = 0; m < M; ++m) {
            const float* v = fields + (uint64_t)m * n;
            float a = INFINITY, hb = -INFINITY;
            for (uint64_t c = b; c < e; ++c) {
                if (v[c] < a) a = v[c];
                if (v[c] > hb) hb = v[c];
            }
            part[(size_t)t * 32 + m] = a;
            part[(size_t)t * 32 + 16 + m] = hb;
        }
        int ml = 0;
        for (uint64_t c = b; c < e; ++c)
            if (level[c] > ml) ml = level[c];
        plev[t] = ml;
    }
    float lo[16], s[16], dmin[16], dmax[16];
    int max_level = 0;
    for (uint32_t m = 0; m < M; ++m) {
        float a = INFINITY, hb = -INFINITY;
        for (int t = 0; t < nt; ++t) {
            if (part[(size_t)t * 32 + m] < a) a = part[(size_t)t * 32 + m];
            if (part[(size_t)t * 32 + 16 + m] > hb) hb = part[(size_t)t * 32 + 16 + m];
        }
        if (n == 0) { a = 0.0f; hb = 0.0f; }
        dmin[m] = a;
        dmax[m] = hb;
        float l = dom_lo[m], h = dom_hi[m];
        if (isnan(l) && isnan(h)) { l = a; h = hb; }
        lo[m] = l;
        s[m] = norm_scale(l, h);
    }
    for (int t = 0; t < nt; ++t)
        if (plev[t] > max_level) max_level = plev[t];

    /* max V: Eq. 5/6 as in orc_update, or the exact maximum over the cells */
    int gi = (int)T - 1, gj = 0;
    for (uint32_t m = 0; m < M; ++m) {
        int im = (int)tf_entry(normalise(dmin[m], lo[m], s[m]), T);
        int jm = (int)tf_entry(normalise(dmax[m], lo[m], s[m]), T);
        if (im < gi) gi = im;
        if (jm > gj) gj = jm;
    }
    if (gi > gj) { gi = 0; gj = 0; }
    float Vmax = 0.0f;
    if (prm->vmax_mode == ORC_VMAX_APPROX) {
        for (int a = gi; a <= gj; ++a) {
            float hi = alpha[a], lw = alpha[a];
            for (uint32_t m = 1; m < M; ++m) {
                float x = alpha[(uint64_t)m * T + a];
                if (x > hi) hi = x;
                if (x < lw) lw = x;
            }
            if (hi - lw > Vmax) Vmax = hi - lw;
        }
    } else {
#pragma omp parallel for num_threads(nt) schedule(static, 1)
        for (int t = 0; t < nt; ++t) {
            uint64_t b, e;
            share(n, nt, t, &b, &e);
            float vm = 0.0f;
            for (uint64_t c = b; c < e; ++c) {
                float hi = 0.0f, lw = 1.0f;
                for (uint32_t m = 0; m < M; ++m) {
                    float al = alpha[(uint64_t)m * T + tf_entry(normalise(fields[(uint64_t)m * n + c], lo[m], s[m]), T)];
                    if (al > hi) hi = al;
                    if (al < lw) lw = al;
                }
                if (hi - lw > vm) vm = hi - lw;
            }
            part[(size_t)t * 32] = vm;
        }
        for (int t = 0; t < nt; ++t)
            if (part[(size_t)t * 32] > Vmax) Vmax = part[(size_t)t * 32];
    }
    free(part);
    free(plev);
    float inv_vmax = Vmax > 0.0f ? 1.0f / Vmax : 0.0f;
    float f_upper = 0.0f;
    int Q = 0;
    if (fixed_point(Vmax, inv_vmax, max_level, n, prm, &f_upper, &Q)) return -5;
    float scale = pow2f_int(Q);

    uint64_t* q = q_out ? q_out : (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint32_t* b1 = b1_out ? b1_out : (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t* b2 = b2_out ? b2_out : (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    u128* tot = (u128*)malloc(sizeof(u128) * (size_t)nt);
    int rc = -3;
    if (!q || !b1 || !b2 || !tot) goto done;

    /* widths (Eq. 1, Eq. 3, fixed point) and per-range totals */
#pragma omp parallel for num_threads(nt) schedule(static, 1)
    for (int t = 0; t < nt; ++t) {
        uint64_t b, e;
        share(n, nt, t, &b, &e);
        u128 acc = 0;
        for (uint64_t c = b; c < e; ++c) {
            float hi = 0.0f, lw = 1.0f;
            for (uint32_t m = 0; m < M; ++m) {
                float tv = normalise(fields[(uint64_t)m * n + c], lo[m], s[m]);
                float al = alpha[(uint64_t)m * T + tf_entry(tv, T)];
                if (al > hi) hi = al;
                if (al < lw) lw = al;
            }
            float f = importance(hi - lw, inv_vmax, level[c], prm);
            q[c] = (uint64_t)nearbyintf(f * scale);
            acc += q[c];
        }
        tot[t] = acc;
    }
    u128 F = 0;
    for (int t = 0; t < nt; ++t) F += tot[t];
    int linear = 0;
    if (F == 0 && n > 0) {
        linear = 1;
#pragma omp parallel for num_threads(nt) schedule(static)
        for (uint64_t c = 0; c < n; ++c) q[c] = 1;
        F = n;
        for (int t = 0; t < nt; ++t) {
            uint64_t b, e;
            share(n, nt, t, &b, &e);
            tot[t] = e - b;
        }
    }
    /* Eq. 4 prefix: exclusive prefix of the range totals, then b1/b2 per cell */
    {
        u128 run = 0;
        for (int t = 0; t < nt; ++t) { u128 x = tot[t]; tot[t] = run; run += x; }
    }
#pragma omp parallel for num_threads(nt) schedule(static, 1)
    for (int t = 0; t < nt; ++t) {
        uint64_t b, e;
        share(n, nt, t, &b, &e);
        u128 E = tot[t];
        for (uint64_t c = b; c < e; ++c) {
            u128 I = E + q[c];
            u128 x1 = E * W / F;
            u128 x2 = I > E ? (I * W + F - 1) / F - 1 : x1;
            if (x1 > W - 1) x1 = W - 1;
            if (x2 > W - 1) x2 = W - 1;
            b1[c] = (uint32_t)x1;
            b2[c] = (uint32_t)x2;
            E = I;
        }
    }

    /* bins: thread t owns pixels [p0, p1) and the run of cells touching them */
    for (uint64_t k = 0; k < (uint64_t)M * W; ++k) { sum[k] = 0.0; vmin[k] = INFINITY; vmax[k] = -INFINITY; }
    for (uint32_t k = 0; k < W; ++k) count[k] = 0;
#pragma omp parallel for num_threads(nt) schedule(static, 1)
    for (int t = 0; t < nt; ++t) {
        uint64_t pb, pe;
        share(W, nt, t, &pb, &pe);
        if (pb == pe) continue;
        uint64_t lo_c = 0, hi_c = n;             /* first cell with b2 >= pb */
        while (lo_c < hi_c) {
            uint64_t mid = lo_c + (hi_c - lo_c) / 2;
            if (b2[mid] < pb) lo_c = mid + 1; else hi_c = mid;
        }
        for (uint64_t c = lo_c; c < n && b1[c] < pe; ++c) {
            uint32_t p0 = b1[c] > pb ? b1[c] : (uint32_t)pb;
            uint32_t p1 = b2[c] < pe - 1 ? b2[c] : (uint32_t)(pe - 1);
            for (uint32_t p = p0; p <= p1; ++p) {
                count[p] += 1;
                for (uint32_t m = 0; m < M; ++m) {
                    float tv = normalise(fields[(uint64_t)m * n + c], lo[m], s[m]);
                    uint64_t k = (uint64_t)m * W + p;
                    sum[k] += (double)tv;
                    if (tv < vmin[k]) vmin[k] = tv;
                    if (tv > vmax[k]) vmax[k] = tv;
                }
            }
        }
    }
    for (uint32_t m = 0; m < M; ++m)
        for (uint32_t p = 0; p < W; ++p) {
            uint64_t k = (uint64_t)m * W + p;
            double mu = count[p] ? sum[k] / (double)count[p] : 0.0;
            float mf = (float)mu;
            if (mean64) mean64[k] = mu;
            if (mean) mean[k] = mf;
            if (y) y[k] = count[p] ? alpha[(uint64_t)m * T + tf_entry(mf, T)] : 0.0f;
            if (!count[p]) { vmin[k] = 0.0f; vmax[k] = 0.0f; }
        }
    if (st) {
        st->vmax = Vmax;
        st->inv_vmax = inv_vmax;
        st->f_upper = f_upper;
        st->Q = Q;
        st->i = gi;
        st->j = gj;
        st->linear = linear;
        st->pow_exact = pow_is_exact(prm->P);
        st->F = (uint64_t)F;
    }
    rc = 0;
done:
    if (!q_out) free(q);
    if (!b1_out) free(b1);
    if (!b2_out) free(b2);
    free(tot);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Gradient of the per-pixel mean alpha w.r.t. alpha control points          */
/* ------------------------------------------------------------------------- */

/* Table entry e interpolates the control points linearly at e/(T-1), control
 * point k sitting at k/(K-1).  Float32 sequence (used for the forward pass
 * that fixes the bin assignment): x = e(K-1)/(T-1), k0 = floor(x),
 * w = x - k0, A = c0 + w (c1 - c0). */
static void ctrl_to_table(uint32_t T, uint32_t K, const float* ctrl, float* table)
{
    for (uint32_t e = 0; e < T; ++e) {
        float x = (float)(e * (K - 1)) / (float)(T - 1);
        uint32_t k0 = (uint32_t)floorf(x);
        if (k0 > K - 2) k0 = K - 2;
        float w = x - (float)k0;
        float c0 = ctrl[k0], c1 = ctrl[k0 + 1];
        table[e] = c0 + w * (c1 - c0);
    }
}

int orc_alpha_grad(uint64_t n, uint32_t M, const float* fields, const uint8_t* level,
                   uint32_t T, uint32_t K, const float* ctrl, const float* dom_lo,
                   const float* dom_hi, const orc_params* prm, const double* target,
                   const double* g_in, double* abar, double* grad, double* loss)
{
    const uint32_t W = prm->width;
    if (K < 2 || M < 1 || M > 16 || T < 2) return -1;
    float* table = (float*)malloc(sizeof(float) * M * T);
    double* sum = (double*)malloc(sizeof(double) * M * W);
    float* vmn = (float*)malloc(sizeof(float) * M * W);
    float* vmx = (float*)malloc(sizeof(float) * M * W);
    uint32_t* cnt = (uint32_t*)malloc(sizeof(uint32_t) * W);
    uint32_t* b1 = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t* b2 = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    double* gtab = (double*)calloc((size_t)M * T, sizeof(double));
    int rc = -3;
    if (!table || !sum || !vmn || !vmx || !cnt || !b1 || !b2 || !gtab) goto done;
    for (uint64_t k = 0; k < (uint64_t)M * K; ++k)
        if (!(ctrl[k] >= 0.0f && ctrl[k] <= 1.0f)) { rc = -1; goto done; }
    /* the interpolated table stays in [0, 1] when the control points do */
    for (uint32_t m = 0; m < M; ++m) ctrl_to_table(T, K, ctrl + (uint64_t)m * K, table + (uint64_t)m * T);
    /* forward: fixes the assignment b1..b2 of every cell */
    rc = orc_update(n, M, fields, level, T, table, dom_lo, dom_hi, prm, sum, vmn, vmx, NULL,
                    NULL, NULL, cnt, NULL, b1, b2, NULL);
    if (rc) goto done;

    float lo[16], s[16];
    for (uint32_t m = 0; m < M; ++m) {
        const float* v = fields + (uint64_t)m * n;
        float a = INFINITY, b = -INFINITY;
        for (uint64_t c = 0; c < n; ++c) { if (v[c] < a) a = v[c]; if (v[c] > b) b = v[c]; }
        float l = dom_lo[m], h = dom_hi[m];
        if (isnan(l) && isnan(h)) { l = a; h = b; }
        lo[m] = l;
        s[m] = norm_scale(l, h);
    }
    /* abar[m][p]: mean over the covering cells of the alpha of the cell's
     * entry, with the table taken in double from the control points. */
    for (uint64_t k = 0; k < (uint64_t)M * W; ++k) abar[k] = 0.0;
    double* tab64 = (double*)malloc(sizeof(double) * M * T);
    if (!tab64) { rc = -3; goto done; }
    for (uint32_t m = 0; m < M; ++m)
        for (uint32_t e = 0; e < T; ++e) {
            double x = (double)e * (double)(K - 1) / (double)(T - 1);
            uint32_t k0 = (uint32_t)floor(x);
            if (k0 > K - 2) k0 = K - 2;
            double w = x - k0;
            tab64[(uint64_t)m * T + e] = (1.0 - w) * ctrl[(uint64_t)m * K + k0] + w * ctrl[(uint64_t)m * K + k0 + 1];
        }
    for (uint64_t c = 0; c < n; ++c)
        for (uint32_t p = b1[c]; p <= b2[c]; ++p)
            for (uint32_t m = 0; m < M; ++m) {
                uint32_t e = tf_entry(normalise(fields[(uint64_t)m * n + c], lo[m], s[m]), T);
                abar[(uint64_t)m * W + p] += tab64[(uint64_t)m * T + e];
            }
    double L = 0.0;
    for (uint32_t m = 0; m < M; ++m)
        for (uint32_t p = 0; p < W; ++p) {
            uint64_t k = (uint64_t)m * W + p;
            abar[k] = cnt[p] ? abar[k] / cnt[p] : 0.0;
            double d = abar[k] - target[k];
            L += d * d;
        }
    /* adjoint: dL/dA_m[e] = sum over covering (cell, pixel) of g/count, with
     * g = dL/dabar = 2 (abar - target), or the caller's g_in when given */
    for (uint64_t c = 0; c < n; ++c)
        for (uint32_t p = b1[c]; p <= b2[c]; ++p)
            for (uint32_t m = 0; m < M; ++m) {
                uint32_t e = tf_entry(normalise(fields[(uint64_t)m * n + c], lo[m], s[m]), T);
                uint64_t k = (uint64_t)m * W + p;
                double gk = g_in ? g_in[k] : 2.0 * (abar[k] - target[k]);
                gtab[(uint64_t)m * T + e] += gk / cnt[p];
            }
    /* chain rule through the linear interpolation of the control points */
    for (uint64_t k = 0; k < (uint64_t)M * K; ++k) grad[k] = 0.0;
    for (uint32_t m = 0; m < M; ++m)
        for (uint32_t e = 0; e < T; ++e) {
            double x = (double)e * (double)(K - 1) / (double)(T - 1);
            uint32_t k0 = (uint32_t)floor(x);
            if (k0 > K - 2) k0 = K - 2;
            double w = x - k0, g = gtab[(uint64_t)m * T + e];
            grad[(uint64_t)m * K + k0] += (1.0 - w) * g;
            grad[(uint64_t)m * K + k0 + 1] += w * g;
        }
    *loss = L;
    free(tab64);
    rc = 0;
done:
    free(table); free(sum); free(vmn); free(vmx); free(cnt); free(b1); free(b2); free(gtab);
    return rc;
}

/* ---- line-plot rasterisation (see dvl_oracle.h) ---------------------------- */

static int32_t plot_row(float v, uint32_t H)
{
    float d = 1.0f - v;                       /* correctly rounded float32 steps */
    float x = d * (float)(H - 1);
    float y = x + 0.5f;
    int32_t r = (int32_t)floorf(y);
    if (r < 0) r = 0;
    if (r > (int32_t)H - 1) r = (int32_t)H - 1;
    return r;
}

int orc_rasterize(uint32_t M, uint32_t W, uint32_t H, const float* values, uint32_t bar_field,
                  uint8_t* lines, uint8_t* bars)
{
    if (M < 1 || M > 8 || W < 1 || H < 1 || !values || bar_field >= M) return -1;
    for (uint64_t i = 0; i < (uint64_t)H * W; ++i) {
        if (lines) lines[i] = 0;
        if (bars) bars[i] = 0;
    }
    for (uint32_t m = 0; m < M; ++m)
        for (uint32_t p = 0; p < W; ++p) {
            const int32_t r = plot_row(values[(uint64_t)m * W + p], H);
            int32_t lo = r, hi = r;
            if (p > 0) {                          /* this column's share of the segment from p-1 */
                const int32_t a = r - (r - plot_row(values[(uint64_t)m * W + p - 1], H)) / 2;
                if (a < lo) lo = a;
                if (a > hi) hi = a;
            }
            if (p + 1 < W) {                      /* and of the segment to p+1 */
                const int32_t b = r + (plot_row(values[(uint64_t)m * W + p + 1], H) - r) / 2;
                if (b < lo) lo = b;
                if (b > hi) hi = b;
            }
            if (lines)
                for (int32_t row = lo; row <= hi; ++row) lines[(uint64_t)row * W + p] |= (uint8_t)(1u << m);
            if (bars && m == bar_field)
                for (int32_t row = r; row < (int32_t)H; ++row) bars[(uint64_t)row * W + p] = 1;
        }
    return 0;
}

/* ---- brushing and linking (see dvl_oracle.h) ------------------------------- */

int orc_brush(uint64_t n, const uint32_t* b1, const uint32_t* b2, uint32_t p0, uint32_t p1, uint64_t* first,
              uint64_t* last)
{
    if (!b1 || !b2 || !first || !last || p0 > p1) return -1;
    uint64_t cnt = 0, f = 0, l = 0;
    for (uint64_t c = 0; c < n; ++c)
        if (b1[c] <= p1 && b2[c] >= p0) {
            if (cnt == 0) f = c;
            l = c;
            ++cnt;
        }
    if (cnt == 0) return 1;
    *first = f;
    *last = l;
    return cnt == l - f + 1 ? 0 : -2;
}

void orc_select_keys(uint64_t n, const uint64_t* keys, uint32_t R, const uint64_t* ranges, uint8_t* mask)
{
    for (uint64_t c = 0; c < n; ++c) {
        uint8_t sel = 0;
        for (uint32_t r = 0; r < R; ++r)
            if (keys[c] >= ranges[2 * r] && keys[c] <= ranges[2 * r + 1]) sel = 1;
        mask[c] = sel;
    }
}

/* ---- widths of sampled cells (see dvl_oracle.h) ------------------------------ */

int orc_widths(uint64_t n_total, uint32_t M, const float* dmin, const float* dmax, uint32_t max_level, uint32_t T,
               const float* alpha, const orc_params* prm, uint64_t k, const float* values, const uint8_t* level,
               uint64_t* q, int32_t* Q_out, float* vmax_out)
{
    if (M < 1 || M > 16 || T < 2 || prm->vmax_mode != ORC_VMAX_APPROX) return -1;
    float lo[16], s[16];
    for (uint32_t m = 0; m < M; ++m) {                 /* default domain: the data range */
        lo[m] = dmin[m];
        s[m] = norm_scale(dmin[m], dmax[m]);
    }
    int gi = (int)T - 1, gj = 0;                        /* Eq. 5 */
    for (uint32_t m = 0; m < M; ++m) {
        int im = (int)tf_entry(normalise(dmin[m], lo[m], s[m]), T);
        int jm = (int)tf_entry(normalise(dmax[m], lo[m], s[m]), T);
        if (im < gi) gi = im;
        if (jm > gj) gj = jm;
    }
    if (gi > gj) { gi = 0; gj = 0; }
    float Vmax = 0.0f;                                  /* Eq. 6 */
    for (int a = gi; a <= gj; ++a) {
        float hi = alpha[a], lw = alpha[a];
        for (uint32_t m = 1; m < M; ++m) {
            float x = alpha[(uint64_t)m * T + a];
            if (x > hi) hi = x;
            if (x < lw) lw = x;
        }
        if (hi - lw > Vmax) Vmax = hi - lw;
    }
    float inv_vmax = Vmax > 0.0f ? 1.0f / Vmax : 0.0f;
    float f_upper = 0.0f;
    int Q = 0;
    if (fixed_point(Vmax, inv_vmax, (int)max_level, n_total, prm, &f_upper, &Q)) return -5;
    float scale = pow2f_int(Q);
    for (uint64_t c = 0; c < k; ++c) {
        float hi = 0.0f, lw = 1.0f;
        for (uint32_t m = 0; m < M; ++m) {
            float t = normalise(values[(uint64_t)m * k + c], lo[m], s[m]);
            float al = alpha[(uint64_t)m * T + tf_entry(t, T)];
            if (al > hi) hi = al;
            if (al < lw) lw = al;
        }
        float f = importance(hi - lw, inv_vmax, level[c], prm);
        q[c] = (uint64_t)nearbyintf(f * scale);
    }
    if (Q_out) *Q_out = Q;
    if (vmax_out) *vmax_out = Vmax;
    return 0;
}

/* ---- log10 value scale (see dvl_oracle.h) ----------------------------------- */

float orc_log10f(float x)
{
    /* c_k = 2 log10(e) / (2k + 1), k = 0..4, rounded to float32 */
    const float c0 = 0x1.bcb7b2p-1f, c1 = 0x1.287a76p-2f, c2 = 0x1.63c628p-3f, c3 = 0x1.fc3fa6p-4f,
                c4 = 0x1.8b4df2p-4f;
    const float l2_hi = 0x1.344p-2f;        /* log10(2) to 16 bits: e * l2_hi is exact */
    const float l2_lo = 0x1.3509f8p-18f;    /* float32(log10(2) - l2_hi) */
    const float s2 = 0x1.6a09e6p+0f;        /* float32(sqrt 2) */
    int e = 0;
    if (x < 0x1p-126f) { x = x * 0x1p24f; e = -24; }   /* subnormal: exact rescale */
    uint32_t b;
    memcpy(&b, &x, 4);
    e += (int)(b >> 23) - 127;
    b = (b & 0x007FFFFFu) | 0x3F800000u;               /* m in [1, 2) */
    float m;
    memcpy(&m, &b, 4);
    if (m >= s2) { m = m * 0.5f; e += 1; }              /* m in [s2/2, s2) */
    const float num = m - 1.0f;                         /* exact (Sterbenz) */
    const float den = m + 1.0f;                         /* rounded ... */
    const float dlo = m - (den - 1.0f);                 /* ... and its exact error: m + 1 = den + dlo */
    const float z = num / den;
    /* z's residual against the exact quotient num / (m + 1):
     * num - z (den + dlo), the first product exact through the fma */
    float r = fmaf(-z, den, num);
    r = fmaf(-z, dlo, r);
    const float dz = r / den;                           /* z + dz = num / (m + 1) to ~2^-48 */
    const float w = z * z;
    float p = c4;
    p = fmaf(p, w, c3);
    p = fmaf(p, w, c2);
    p = fmaf(p, w, c1);
    p = fmaf(p, w, c0);
    const float lm = fmaf(z, p, dz * c0);               /* log10 m = (z + dz) p */
    const float ef = (float)e;
    return fmaf(ef, l2_hi, fmaf(ef, l2_lo, lm));
}

int orc_log_field(uint64_t n, float* v)
{
    float pos = 0.0f;                  /* smallest positive value */
    for (uint64_t i = 0; i < n; ++i)
        if (v[i] > 0.0f && (pos == 0.0f || v[i] < pos)) pos = v[i];
    if (!(pos > 0.0f)) return -5;
    for (uint64_t i = 0; i < n; ++i) v[i] = orc_log10f(v[i] > 0.0f ? v[i] : pos);
    return 0;
}
