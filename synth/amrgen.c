/*
 * Seeded synthetic multi-field AMR generator (input data only).
 *
 * This module produces the INPUTS of the dynamic-volume-line computation: AMR
 * cells given by their lower corner on the logical grid plus their refinement
 * level (0 = finest, cell width 2^L; paper Sec. 2.1) and four correlated scalar
 * fields shaped like the paper's astrophysics data (dens, temp, pres, velmag;
 * paper Sec. 6).  It contains none of the method's arithmetic: no space-filling
 * curve, no transfer function, no importance, no binning.  Both the CPU oracle
 * and the CUDA path consume its output; neither is used here.
 *
 * Randomness is counter based: every lattice value is splitmix64 (Steele, Lea,
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) of a
 * key built from (seed, stream, octave, i, j, k), so any cell can be
 * regenerated in isolation and the output does not depend on the thread count.
 *
 * Fields are smooth 3D value noise (trilinear interpolation of lattice values
 * with a smoothstep fade, 4 octaves, lacunarity 2, gain 0.5), evaluated in
 * double precision at each cell's centroid and stored as float:
 *   dens   = exp(MU_D + SIG_D * n1)                          (log-normal)
 *   temp   = exp(MU_T + SIG_T * (RHO * n1 + sqrt(1-RHO^2) * n2))  (log-normal,
 *            anti-correlated with density)
 *   pres   = dens * temp
 *   velmag = |MU_V + SIG_V * n3|                              (|Gaussian|)
 *
 * Two structure modes:
 *   mode 0 (threshold): a base grid of base_n^3 cells at level n_levels-1; a
 *     cell of level L > 0 is split into its 8 children when the density noise
 *     n1 at its centroid exceeds tau.  Cells are emitted base cell by base cell
 *     (z slowest, x fastest), depth first, children in z/y/x order.
 *   mode 1 (bricks): base_n^3 cells at level 1 grouped into bricks of
 *     brick^3 base cells; n_refined seeded bricks are split once (level 0).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define MU_D 0.0
#define SIG_D 1.5
#define MU_T 4.0
#define SIG_T 0.8
#define RHO (-0.6)
#define MU_V 1.0
#define SIG_V 1.0
#define OCTAVES 4
#define BASE_FREQ 4.0   /* lattice cells across the domain at octave 0 */
/* Divides the octave sum so that n has roughly unit standard deviation
 * (measured once on 2^20 random points). */
#define NOISE_NORM 0.43

typedef struct {
    int32_t mode;          /* 0 threshold refinement, 1 bricks */
    int32_t base_n;        /* base cells per dimension */
    int32_t n_levels;      /* levels n_levels-1 (base) .. 0 */
    int32_t brick;         /* mode 1: brick edge in base cells */
    int32_t n_refined;     /* mode 1: number of refined bricks */
    int32_t n_threads;     /* 0 = all online cores */
    double tau;            /* mode 0: refine when n1 > tau */
    uint64_t seed;
    int32_t box_lo[3];     /* mode 0: only base cells in [box_lo, box_lo + box_n)^3 */
    int32_t box_n;         /* 0 = the whole base grid */
} amrgen_cfg;

static inline uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline double lattice(uint64_t key, int64_t i, int64_t j, int64_t k)
{
    uint64_t h = splitmix64(key + (uint64_t)i);
    h = splitmix64(h + (uint64_t)j);
    h = splitmix64(h + (uint64_t)k);
    return (double)(h >> 11) * 0x1.0p-53 * 2.0 - 1.0;
}

static inline double fade(double t) { return t * t * (3.0 - 2.0 * t); }

/* value noise at p (domain units, [0,1)^3) for the given stream */
static double noise(uint64_t seed, int stream, const double p[3])
{
    double sum = 0.0, amp = 1.0, freq = BASE_FREQ;
    for (int o = 0; o < OCTAVES; ++o) {
        uint64_t key = splitmix64(seed * 0x100000001B3ull + (uint64_t)(stream * 16 + o));
        double x = p[0] * freq, y = p[1] * freq, z = p[2] * freq;
        double fx = floor(x), fy = floor(y), fz = floor(z);
        int64_t i = (int64_t)fx, j = (int64_t)fy, k = (int64_t)fz;
        double u = fade(x - fx), v = fade(y - fy), w = fade(z - fz);
        double c000 = lattice(key, i, j, k), c100 = lattice(key, i + 1, j, k);
        double c010 = lattice(key, i, j + 1, k), c110 = lattice(key, i + 1, j + 1, k);
        double c001 = lattice(key, i, j, k + 1), c101 = lattice(key, i + 1, j, k + 1);
        double c011 = lattice(key, i, j + 1, k + 1), c111 = lattice(key, i + 1, j + 1, k + 1);
        double x00 = c000 + u * (c100 - c000), x10 = c010 + u * (c110 - c010);
        double x01 = c001 + u * (c101 - c001), x11 = c011 + u * (c111 - c011);
        double y0 = x00 + v * (x10 - x00), y1 = x01 + v * (x11 - x01);
        sum += amp * (y0 + w * (y1 - y0));
        amp *= 0.5;
        freq *= 2.0;
    }
    return sum / NOISE_NORM;
}

static inline int64_t grid_extent(const amrgen_cfg* c)
{
    return (int64_t)c->base_n << (c->n_levels - 1);
}

static inline void centroid(const amrgen_cfg* c, const int32_t lo[3], int level, double p[3])
{
    double G = (double)grid_extent(c);
    double half = (double)(1 << level) * 0.5;
    for (int d = 0; d < 3; ++d) p[d] = ((double)lo[d] + half) / G;
}

static void cell_fields(const amrgen_cfg* c, const double p[3], double n1, float out[4])
{
    double n2 = noise(c->seed, 1, p), n3 = noise(c->seed, 2, p);
    double dens = exp(MU_D + SIG_D * n1);
    double temp = exp(MU_T + SIG_T * (RHO * n1 + sqrt(1.0 - RHO * RHO) * n2));
    out[0] = (float)dens;
    out[1] = (float)temp;
    out[2] = (float)(dens * temp);
    out[3] = (float)fabs(MU_V + SIG_V * n3);
}

/* ---------------- mode 0: threshold refinement ---------------- */

typedef struct {
    int32_t *lx, *ly, *lz;
    uint8_t* level;
    float *f0, *f1, *f2, *f3;
    int64_t pos;
    int count_only;
} sink;

static void visit(const amrgen_cfg* c, int32_t lx, int32_t ly, int32_t lz, int level, sink* s)
{
    int32_t lo[3] = {lx, ly, lz};
    double p[3];
    centroid(c, lo, level, p);
    double n1 = noise(c->seed, 0, p);
    if (level > 0 && n1 > c->tau) {
        int32_t h = 1 << (level - 1);
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                    visit(c, lx + dx * h, ly + dy * h, lz + dz * h, level - 1, s);
        return;
    }
    if (!s->count_only) {
        float f[4];
        cell_fields(c, p, n1, f);
        int64_t i = s->pos;
        s->lx[i] = lx; s->ly[i] = ly; s->lz[i] = lz;
        s->level[i] = (uint8_t)level;
        s->f0[i] = f[0]; s->f1[i] = f[1]; s->f2[i] = f[2]; s->f3[i] = f[3];
    }
    s->pos++;
}

/* b-th base cell of the selected box (z slowest, x fastest) */
static void base_cell(const amrgen_cfg* c, int64_t b, int32_t xyz[3])
{
    int64_t n = c->box_n > 0 ? c->box_n : c->base_n;
    xyz[0] = (int32_t)(b % n);
    xyz[1] = (int32_t)((b / n) % n);
    xyz[2] = (int32_t)(b / (n * n));
    if (c->box_n > 0)
        for (int d = 0; d < 3; ++d) xyz[d] += c->box_lo[d];
}

static int64_t n_base(const amrgen_cfg* c)
{
    int64_t n = c->box_n > 0 ? c->box_n : c->base_n;
    return n * n * n;
}

typedef struct {
    const amrgen_cfg* c;
    int64_t b0, b1, stride;     /* base cells b0, b0+stride, ... < b1 */
    uint32_t* counts;           /* per base cell (count pass) or NULL */
    const int64_t* offsets;     /* per base cell (fill pass) or NULL */
    sink out;
    int64_t total;
} job;

static void* run_job(void* arg)
{
    job* J = (job*)arg;
    const amrgen_cfg* c = J->c;
    int32_t level = c->n_levels - 1, w = 1 << level;
    J->total = 0;
    for (int64_t b = J->b0; b < J->b1; b += J->stride) {
        int32_t xyz[3];
        base_cell(c, b, xyz);
        sink s = J->out;
        s.count_only = (J->offsets == NULL);
        s.pos = s.count_only ? 0 : J->offsets[b];
        int64_t start = s.pos;
        visit(c, xyz[0] * w, xyz[1] * w, xyz[2] * w, level, &s);
        int64_t cnt = s.pos - start;
        if (J->counts) J->counts[b] = (uint32_t)cnt;
        J->total += cnt;
    }
    return NULL;
}

static int threads_for(const amrgen_cfg* c)
{
    int t = c->n_threads;
    if (t <= 0) {
        long n = sysconf(_SC_NPROCESSORS_ONLN);
        t = n > 0 ? (int)n : 1;
    }
    if (t > 256) t = 256;
    return t;
}

/* Runs base cells {offset, offset+stride, ...} split across threads. */
static int64_t run_parallel(const amrgen_cfg* c, int64_t stride, int64_t offset,
                            uint32_t* counts, const int64_t* offsets, const sink* out)
{
    int64_t nb = n_base(c);
    int64_t nsel = nb > offset ? (nb - offset + stride - 1) / stride : 0;
    int T = threads_for(c);
    if (nsel < T) T = nsel > 0 ? (int)nsel : 1;
    job jobs[256];
    pthread_t th[256];
    int64_t per = (nsel + T - 1) / T;
    for (int t = 0; t < T; ++t) {
        int64_t s0 = t * per, s1 = (t + 1) * per;
        if (s1 > nsel) s1 = nsel;
        jobs[t].c = c;
        jobs[t].b0 = offset + s0 * stride;
        jobs[t].b1 = s1 > s0 ? offset + s1 * stride : jobs[t].b0;
        if (jobs[t].b1 > nb) jobs[t].b1 = nb;
        jobs[t].stride = stride;
        jobs[t].counts = counts;
        jobs[t].offsets = offsets;
        if (out) jobs[t].out = *out; else memset(&jobs[t].out, 0, sizeof(sink));
        if (T > 1) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    }
    int64_t total = 0;
    if (T == 1) run_job(&jobs[0]);
    for (int t = 0; t < T; ++t) {
        if (T > 1) pthread_join(th[t], NULL);
        total += jobs[t].total;
    }
    return total;
}

/* Number of leaf cells over the base cells offset, offset+stride, ... */
int64_t amrgen_count_sample(const amrgen_cfg* c, int64_t stride, int64_t offset)
{
    if (c->mode != 0 || stride < 1 || offset < 0) return -1;
    return run_parallel(c, stride, offset, NULL, NULL, NULL);
}

/* Per-base-cell leaf counts (length base_n^3); returns the total. */
int64_t amrgen_count(const amrgen_cfg* c, uint32_t* counts)
{
    if (c->mode != 0) return -1;
    return run_parallel(c, 1, 0, counts, NULL, NULL);
}

/* Fills the cells; offsets[b] = first output index of base cell b. */
int amrgen_fill(const amrgen_cfg* c, const int64_t* offsets, int32_t* lx, int32_t* ly,
                int32_t* lz, uint8_t* level, float* f0, float* f1, float* f2, float* f3)
{
    if (c->mode != 0) return -1;
    sink s = {lx, ly, lz, level, f0, f1, f2, f3, 0, 0};
    run_parallel(c, 1, 0, NULL, offsets, &s);
    return 0;
}

/* ---------------- mode 1: bricks ---------------- */

int64_t amrgen_bricks_count(const amrgen_cfg* c)
{
    int64_t nb = c->base_n / c->brick;
    int64_t bricks = nb * nb * nb, bc = (int64_t)c->brick * c->brick * c->brick;
    if (c->mode != 1 || c->n_levels != 2 || c->base_n % c->brick || c->n_refined > bricks) return -1;
    return (bricks - c->n_refined) * bc + (int64_t)c->n_refined * bc * 8;
}

int amrgen_bricks_fill(const amrgen_cfg* c, int32_t* lx, int32_t* ly, int32_t* lz, uint8_t* level,
                       float* f0, float* f1, float* f2, float* f3)
{
    if (amrgen_bricks_count(c) < 0) return -1;
    int32_t nb = c->base_n / c->brick, bricks = nb * nb * nb;
    uint8_t* refined = (uint8_t*)calloc((size_t)bricks, 1);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)bricks);
    if (!refined || !order) { free(refined); free(order); return -2; }
    /* seeded partial Fisher-Yates: the first n_refined entries are refined */
    for (int32_t i = 0; i < bricks; ++i) order[i] = i;
    uint64_t st = c->seed ^ 0xB41C5ull;
    for (int32_t i = 0; i < c->n_refined; ++i) {
        st = splitmix64(st);
        int32_t j = i + (int32_t)(st % (uint64_t)(bricks - i));
        int32_t tmp = order[i]; order[i] = order[j]; order[j] = tmp;
        refined[order[i]] = 1;
    }
    int64_t pos = 0;
    for (int32_t b = 0; b < bricks; ++b) {
        int32_t bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
        int lvl = refined[b] ? 0 : 1;
        int32_t w = 1 << lvl;                 /* cell width on the logical grid */
        int32_t e = c->brick * 2 / w;         /* cells per brick edge */
        int32_t ox = bx * c->brick * 2, oy = by * c->brick * 2, oz = bz * c->brick * 2;
        for (int32_t z = 0; z < e; ++z)
            for (int32_t y = 0; y < e; ++y)
                for (int32_t x = 0; x < e; ++x) {
                    int32_t lo[3] = {ox + x * w, oy + y * w, oz + z * w};
                    double p[3];
                    centroid(c, lo, lvl, p);
                    float f[4];
                    cell_fields(c, p, noise(c->seed, 0, p), f);
                    lx[pos] = lo[0]; ly[pos] = lo[1]; lz[pos] = lo[2];
                    level[pos] = (uint8_t)lvl;
                    f0[pos] = f[0]; f1[pos] = f[1]; f2[pos] = f[2]; f3[pos] = f[3];
                    pos++;
                }
    }
    free(refined);
    free(order);
    return 0;
}

/* Density noise n1 at arbitrary points (domain units), for tests of the
 * generator's statistics. */
void amrgen_noise(uint64_t seed, int stream, int64_t n, const double* xyz, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = noise(seed, stream, xyz + 3 * i);
}
