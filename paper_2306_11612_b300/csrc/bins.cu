// Per-pixel bins as range queries (paper Sec. 3.2).
//
// In curve order the cells that touch pixel p form one contiguous range
// [lo_p, hi_p] (both the first and the last pixel of a cell's span are
// non-decreasing in the cell index).  The value a cell contributes to the bins
// is its normalised field value t, which does not depend on the transfer
// function.  So, once per data set and TF domain, this file builds value
// tables -- per 128-cell step, the exact fixed-point sum of t and its min/max
// (an exclusive prefix of the sums, and a sparse table of min/max over every
// power-of-two run of steps) -- and each update then needs only:
//   k_bounds  for every pixel boundary j, H(j) = number of cells whose span
//             starts before the boundary's first position C(j), and whether
//             the last of them also reaches pixel j ("straddles"); found by a
//             32-way search over the scan's chunk prefixes and an exact
//             recomputation of the widths of the one step that contains it.
//             It also records the partial-step sums/min/max of the two pixels
//             that meet in that step;
//   k_pixels  for every pixel: count = hi - lo + 1, sums from the prefix
//             table plus the two recorded partial steps, min/max from two
//             sparse-table entries and the records, then mean and the alpha of
//             the mean.
// Sums are exact integer sums of floor(t * 2^95), so the bins do not depend
// on any summation order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cell_math.cuh"
#include "dvl_internal.h"

namespace dvl {

namespace {

typedef unsigned __int128 u128;
constexpr int FX_BITS = 95;          // fixed-point fraction bits of t

// floor(t * 2^95) for 0 <= t <= 1 (t a float32): t = mant * 2^(ex-150), so the
// value is mant shifted left by ex - 150 + 95 (mant < 2^24, shift at most 72).
__device__ __forceinline__ u128 fx_of(float t)
{
    const uint32_t b = __float_as_uint(t);
    const int ex = (int)(b >> 23);                    // t >= +0: no sign bit
    if (ex == 0) return 0;                            // zero or subnormal: below 2^-126
    const uint64_t mant = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = ex - 150 + FX_BITS;
    if (sh < 0) return sh > -24 ? (u128)(mant >> -sh) : (u128)0;
    const uint64_t lo = sh < 64 ? mant << sh : 0ull;
    const uint64_t hi = sh <= 40 ? 0ull : (sh < 64 ? mant >> (64 - sh) : mant << (sh - 64));
    return ((u128)hi << 64) | lo;
}

// Warp sum of per-lane values below 2^120, exact: five 24-bit limbs, each
// summed by one redux (32 x 2^24 < 2^32), then recombined.
__device__ __forceinline__ u128 warp_sum_limbs(u128 x)
{
    u128 r = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const uint32_t limb = (uint32_t)(x >> (24 * k)) & 0xFFFFFFu;
        r += (u128)__reduce_add_sync(FULL, limb) << (24 * k);
    }
    return r;
}

__device__ __forceinline__ double fx_to_double(u128 x)
{
    const double hi = (double)(uint64_t)(x >> 64), lo = (double)(uint64_t)x;
    return (hi * 18446744073709551616.0 + lo) * 0x1.0p-95;
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 x, int o)
{
    const uint64_t lo = __shfl_xor_sync(FULL, (unsigned long long)(uint64_t)x, o);
    const uint64_t hi = __shfl_xor_sync(FULL, (unsigned long long)(uint64_t)(x >> 64), o);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 warp_sum_u128(u128 x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x += shfl_xor_u128(x, o);
    return x;
}

__device__ __forceinline__ float warp_min(float x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fminf(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

__device__ __forceinline__ float warp_max(float x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(FULL, x, o));
    return x;
}

// ---- value tables ------------------------------------------------------------

// One warp per 128-cell step: fixed-point sum, min and max of t per field.
template <int M>
__global__ __launch_bounds__(256) void k_vt_steps(ValueTableArgs v)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    float lo[M], sc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) { lo[m] = v.consts->lo[m]; sc[m] = v.consts->s[m]; }
    for (uint64_t st = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); st < v.n_steps; st += warps) {
        const uint64_t idx = st * STEP + lane * 4;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            u128 sum = 0;
            float mn = 3.0f, mx = -1.0f;
            if (idx < v.n) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(v.val + m * v.pitch + idx));
                const float c[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (idx + j < v.n) {
                        const float t = norm_t(c[j], lo[m], sc[m]);
                        sum += fx_of(t);
                        mn = fminf(mn, t);
                        mx = fmaxf(mx, t);
                    }
            }
            sum = warp_sum_u128(sum);
            mn = warp_min(mn);
            mx = warp_max(mx);
            if (lane == 0) {
                const uint64_t k = (uint64_t)m * (v.n_steps + 1) + st;
                v.pre_lo[k] = (uint64_t)sum;
                v.pre_hi[k] = (uint64_t)(sum >> 64);
                v.mn[(uint64_t)m * v.level_stride + st] = mn;
                v.mx[(uint64_t)m * v.level_stride + st] = mx;
            }
        }
    }
}

// Exclusive scan of the step sums of every field, in blocks of 1024 steps
// (phase 1: in-block scan and block totals; phase 2: scan of the totals;
// phase 3: add the block offsets).  u128 adds are exact and associative.
__global__ __launch_bounds__(256) void k_vt_scan1(ValueTableArgs v, uint64_t* tot_lo, uint64_t* tot_hi)
{
    __shared__ u128 s[256];
    const uint32_t m = blockIdx.y;
    const uint64_t b0 = (uint64_t)blockIdx.x * 1024;
    const uint64_t row = (uint64_t)m * (v.n_steps + 1);
    u128 x[4], acc = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t k = b0 + threadIdx.x * 4 + i;
        x[i] = k < v.n_steps ? (((u128)v.pre_hi[row + k] << 64) | v.pre_lo[row + k]) : (u128)0;
        acc += x[i];
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {            // Hillis-Steele inclusive scan of thread sums
        u128 y = threadIdx.x >= o ? s[threadIdx.x - o] : (u128)0;
        __syncthreads();
        s[threadIdx.x] += y;
        __syncthreads();
    }
    u128 run = s[threadIdx.x] - acc;               // exclusive prefix of this thread
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t k = b0 + threadIdx.x * 4 + i;
        if (k < v.n_steps) {
            v.pre_lo[row + k] = (uint64_t)run;
            v.pre_hi[row + k] = (uint64_t)(run >> 64);
        }
        run += x[i];
    }
    if (threadIdx.x == 255) {
        const uint64_t nb = gridDim.x;
        tot_lo[m * nb + blockIdx.x] = (uint64_t)s[255];
        tot_hi[m * nb + blockIdx.x] = (uint64_t)(s[255] >> 64);
    }
}

__global__ void k_vt_scan2(ValueTableArgs v, uint64_t* tot_lo, uint64_t* tot_hi, uint32_t nb)
{
    if (threadIdx.x != 0) return;
    const uint32_t m = blockIdx.x;
    u128 run = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        const u128 t = ((u128)tot_hi[m * nb + b] << 64) | tot_lo[m * nb + b];
        tot_lo[m * nb + b] = (uint64_t)run;
        tot_hi[m * nb + b] = (uint64_t)(run >> 64);
        run += t;
    }
    const uint64_t row = (uint64_t)m * (v.n_steps + 1);
    v.pre_lo[row + v.n_steps] = (uint64_t)run;           // prefix up to the end
    v.pre_hi[row + v.n_steps] = (uint64_t)(run >> 64);
}

__global__ __launch_bounds__(256) void k_vt_scan3(ValueTableArgs v, const uint64_t* tot_lo, const uint64_t* tot_hi)
{
    const uint32_t m = blockIdx.y;
    const uint64_t nb = gridDim.x;
    const u128 off = ((u128)tot_hi[m * nb + blockIdx.x] << 64) | tot_lo[m * nb + blockIdx.x];
    const uint64_t row = (uint64_t)m * (v.n_steps + 1);
    for (int i = 0; i < 4; ++i) {
        const uint64_t k = (uint64_t)blockIdx.x * 1024 + threadIdx.x * 4 + i;
        if (k < v.n_steps) {
            const u128 x = (((u128)v.pre_hi[row + k] << 64) | v.pre_lo[row + k]) + off;
            v.pre_lo[row + k] = (uint64_t)x;
            v.pre_hi[row + k] = (uint64_t)(x >> 64);
        }
    }
}

// Level l of the min/max sparse table: entry i covers steps [i, i + 2^l)
// (entries whose range would pass the last step are never read).
__global__ void k_vt_level(ValueTableArgs v, int l)
{
    const uint32_t m = blockIdx.y;
    const uint64_t half = 1ull << (l - 1), n = v.n_steps + 1 - 2 * half;   // i + 2^l <= n_steps
    float* mn = v.mn + (uint64_t)m * v.level_stride;
    float* mx = v.mx + (uint64_t)m * v.level_stride;
    const uint64_t prev = (uint64_t)(l - 1) * v.n_steps, cur = (uint64_t)l * v.n_steps;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        mn[cur + i] = fminf(mn[prev + i], mn[prev + i + half]);
        mx[cur + i] = fmaxf(mx[prev + i], mx[prev + i + half]);
    }
}

// ---- queries -------------------------------------------------------------------

// Last chunk whose exclusive width prefix is below X (chunk 0 always is, as
// its prefix is 0 < X): a 32-way search, one probe per lane per round.
__device__ __forceinline__ uint64_t find_chunk(const unsigned long long* prefix, uint64_t n_chunks,
                                               unsigned long long X, int lane)
{
    uint64_t lo = 0, hi = n_chunks - 1;                  // answer in [lo, hi]
    while (hi - lo >= 32) {
        const uint64_t stride = (hi - lo + 32) / 32;     // 32 probes cover [lo, hi]
        const uint64_t at = lo + (uint64_t)lane * stride;
        const bool below = at <= hi && prefix[at] < X;
        const unsigned mask = __ballot_sync(FULL, below);   // lane 0 is always set
        const int last = 31 - __clz(mask);
        const uint64_t nlo = lo + (uint64_t)last * stride;
        const uint64_t nhi = nlo + stride - 1;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    const uint64_t at = lo + lane;
    const unsigned mask = __ballot_sync(FULL, at <= hi && prefix[at] < X);
    return lo + (31 - __clz(mask));
}

// Over the 128-cell step starting at cell stb (cells below ste exist), the
// sums (fixed point), min and max of t of the cells below H ("tail") and of
// the cells from `first` on ("head"), reduced over the warp with redux.  Each
// cell is converted once; min/max work on the bits of t >= 0 (empty: +inf, 0,
// which are neutral for values in [0, 1]).  Written by lane 0 to the records
// of boundary j.
template <int M>
__device__ __forceinline__ void step_partials(const UpdateArgs& a, const UpdateConsts* C, const QueryArgs& qa,
                                              uint32_t j, uint64_t stb, uint64_t ste, uint64_t H, uint64_t first,
                                              int lane)
{
    const uint64_t idx = stb + lane * 4;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const float lo = C->lo[m], sc = C->s[m];
        u128 ts = 0, hs = 0;
        uint32_t tmn = 0x7F800000u, tmx = 0u, hmn = 0x7F800000u, hmx = 0u;
        if (idx < ste) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(a.val + m * a.pitch + idx));
            const float c[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t cell = idx + k;
                const float t = norm_t(c[k], lo, sc);
                const uint32_t tb = __float_as_uint(t);
                const u128 f = fx_of(t);
                if (cell < H) {
                    ts += f;
                    tmn = min(tmn, tb);
                    tmx = max(tmx, tb);
                }
                if (cell >= first && cell < ste) {
                    hs += f;
                    hmn = min(hmn, tb);
                    hmx = max(hmx, tb);
                }
            }
        }
        ts = warp_sum_limbs(ts);
        hs = warp_sum_limbs(hs);
        tmn = __reduce_min_sync(FULL, tmn);
        tmx = __reduce_max_sync(FULL, tmx);
        hmn = __reduce_min_sync(FULL, hmn);
        hmx = __reduce_max_sync(FULL, hmx);
        if (lane == 0) {
            const uint64_t kt = ((uint64_t)j * 2 + 0) * M + m, kh = kt + M;
            qa.psum[kt] = make_ulonglong2((unsigned long long)(uint64_t)ts, (unsigned long long)(uint64_t)(ts >> 64));
            qa.pmm[kt] = make_float2(__uint_as_float(tmn), __uint_as_float(tmx));
            qa.psum[kh] = make_ulonglong2((unsigned long long)(uint64_t)hs, (unsigned long long)(uint64_t)(hs >> 64));
            qa.pmm[kh] = make_float2(__uint_as_float(hmn), __uint_as_float(hmx));
        }
    }
}

// Pixel boundary j in [1, W-1]: H = #cells with span start E < C(j), and
// whether the last of them (cell H-1) has a positive width reaching past the
// real boundary j F / W (then it also touches pixel j).  Also records, over
// the step that holds cell H-1, the partial sums/min/max of pixel j-1's last
// cells and of pixel j's first cells, so that the pixel queries read no
// cells except where a pixel lies inside one step.
template <int M, int PM>
__device__ __forceinline__ void bounds_one(const UpdateArgs& a, const QueryArgs& qa, const float* s_tf, uint32_t j,
                                           int lane)
{
    const UpdateConsts* C = qa.consts;
    const unsigned long long F = C->F;
    const PixelMap pm{F / a.W, F % a.W, F, a.W};
    const unsigned long long X = pm.C(j);
    const u128 jF = (u128)j * F;
    unsigned long long H;
    bool S;
    if (C->linear) {                                      // widths 1: E_c = c
        H = X < a.n ? X : a.n;
        S = H >= 1 && (u128)H * a.W > jF;
    } else {
        const uint64_t n_chunks = (a.n + CHUNK - 1) / CHUNK;
        const uint64_t chunk = find_chunk(qa.chunk_prefix, n_chunks, X, lane), base = chunk * CHUNK;
        const uint64_t rem = a.n - base;
        const int nsteps = rem >= (uint64_t)CHUNK ? STEPS : (int)((rem + STEP - 1) / STEP);
        unsigned long long ssum = lane < nsteps ? qa.step_sums[chunk * STEPS + lane] : 0ull;
        const unsigned long long start = qa.chunk_prefix[chunk] + warp_incl_scan_u64(ssum, lane) - ssum;
        const unsigned before = __ballot_sync(FULL, lane < nsteps && start < X);
        const int st = 31 - __clz(before);                 // last step starting before X
        // exact widths of that step's cells
        Cell<M, PM> cc;
        cc.load(C, a.T);
        const uint64_t idx = base + st * STEP + lane * 4;
        uint32_t q[4] = {0, 0, 0, 0};
        if (idx < a.n) {
            float v[4][M];
            uint32_t L4;
            load4<M>(a.val, a.pitch, a.lev, idx, v, L4);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float t[M];
#pragma unroll
                for (int m = 0; m < M; ++m) t[m] = norm_t(v[c][m], cc.lo[m], cc.s[m]);
                if (idx + c < a.n) q[c] = cc.width(t, (L4 >> (8 * c)) & 0xFF, s_tf);
            }
        }
        const unsigned long long lsum = (unsigned long long)q[0] + q[1] + q[2] + q[3];
        unsigned long long E = __shfl_sync(FULL, start, st) + warp_incl_scan_u64(lsum, lane) - lsum;
        uint32_t cnt = 0;
        unsigned long long lastI = 0;
        bool lastpos = false;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (idx + c < a.n && E < X) {
                ++cnt;
                lastI = E + q[c];
                lastpos = q[c] > 0;
            }
            E += q[c];
        }
        const uint32_t total = __reduce_add_sync(FULL, cnt);
        const unsigned has = __ballot_sync(FULL, cnt > 0);
        const int owner = 31 - __clz(has);                 // lane holding cell H-1
        const unsigned long long I = __shfl_sync(FULL, lastI, owner);
        const bool pos = __shfl_sync(FULL, lastpos, owner);
        H = base + st * STEP + total;
        S = pos && (u128)I * a.W > jF;
    }
    // partial terms over the step of cell H-1 (H >= 1: the step's first cell starts before X)
    const uint64_t stb = (H - 1) / STEP * STEP;
    const uint64_t ste = stb + STEP < a.n ? stb + STEP : a.n;
    step_partials<M>(a, C, qa, j, stb, ste, H, S ? H - 1 : H, lane);
    if (lane == 0) {
        qa.H[j] = H;
        qa.S[j] = S;
    }
}

template <int M, int PM>
__global__ __launch_bounds__(256) void k_bounds(UpdateArgs a, QueryArgs qa)
{
    extern __shared__ float s_tf[];
    load_table<M>(s_tf, a.tf, a.T);
    __syncthreads();
    const uint32_t j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) + 1;
    if (j >= a.W) return;
    bounds_one<M, PM>(a, qa, s_tf, j, threadIdx.x & 31);
}

// Min/max of t over steps [s0, s1) (s0 < s1) of one field: two overlapping
// power-of-two ranges of the sparse table.
__device__ __forceinline__ void steps_minmax(const ValueTableArgs& v, uint32_t m, uint64_t s0, uint64_t s1,
                                             float& mn, float& mx)
{
    const int k = 63 - __clzll((long long)(s1 - s0));
    const uint64_t row = (uint64_t)m * v.level_stride + (uint64_t)k * v.n_steps;
    const uint64_t b = s1 - (1ull << k);
    mn = fminf(mn, fminf(v.mn[row + s0], v.mn[row + b]));
    mx = fmaxf(mx, fmaxf(v.mx[row + s0], v.mx[row + b]));
}

// One thread per pixel: the bins of cells [lo_p, hi_p].  With s_p the step of
// boundary p's cell H(p)-1 and s_q that of boundary p+1, the range is the
// head recorded at boundary p, the whole steps (s_p, s_q) from the value
// tables, and the tail recorded at boundary p+1 (the first pixel starts at
// step 0, the last one ends with the last step).  A pixel inside a single
// step reads its cells directly.
template <int M>
__device__ __forceinline__ void pixels_field(const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v,
                                             uint32_t p, int m)
{
    const bool has_l = p > 0, has_r = p + 1 < a.W;
    const uint64_t bl = (uint64_t)p * qa.hstride, br = (uint64_t)(p + 1) * qa.hstride;   // boundary entries
    const uint64_t Hn = has_r ? qa.H[br] : a.n;                    // cells with E < C(p+1)
    const uint64_t Hp = has_l ? qa.H[bl] : 0;
    const uint64_t lo_c = has_l ? (qa.S[bl] ? Hp - 1 : Hp) : 0;
    const uint64_t k = (uint64_t)m * a.W + p;
    if (Hn == 0 || Hn - 1 < lo_c) {                                  // no cell touches p
        a.sum[k] = 0.0;
        a.vmin[k] = 0u;
        a.vmax[k] = 0u;
        a.mean[k] = 0.0f;
        a.y[k] = 0.0f;
        if (m == 0) a.count[p] = 0u;
        return;
    }
    const uint64_t c1 = Hn;
    const uint32_t count = (uint32_t)(c1 - lo_c);
    const UpdateConsts* C = qa.consts;
    const uint64_t sp = has_l ? (Hp - 1) / STEP : 0, sq = has_r ? (Hn - 1) / STEP : 0;
    const bool one_step = has_l && has_r && sp == sq;
    const uint64_t w0 = has_l ? sp + 1 : 0, w1 = has_r ? sq : v.n_steps;   // whole steps [w0, w1)
    float mn = 3.0f, mx = -1.0f;
    u128 sum = 0;
    if (one_step) {
        const float lo = C->lo[m], sc = C->s[m];
        for (uint64_t c = lo_c; c < c1; ++c) {
            const float t = norm_t(__ldg(a.val + m * a.pitch + c), lo, sc);
            sum += fx_of(t);
            mn = fminf(mn, t);
            mx = fmaxf(mx, t);
        }
    } else {
        if (w1 > w0) {
            steps_minmax(v, m, w0, w1, mn, mx);
            const uint64_t row = (uint64_t)m * (v.n_steps + 1);
            const u128 pa = ((u128)v.pre_hi[row + w0] << 64) | v.pre_lo[row + w0];
            const u128 pb = ((u128)v.pre_hi[row + w1] << 64) | v.pre_lo[row + w1];
            sum = pb - pa;
        }
        if (has_l) {
            const uint64_t q = (bl * 2 + 1) * M + m;
            const ulonglong2 ps = qa.psum[q];
            const float2 mm = qa.pmm[q];
            sum += ((u128)ps.y << 64) | ps.x;
            mn = fminf(mn, mm.x);
            mx = fmaxf(mx, mm.y);
        }
        if (has_r) {
            const uint64_t q = (br * 2 + 0) * M + m;
            const ulonglong2 ps = qa.psum[q];
            const float2 mm = qa.pmm[q];
            sum += ((u128)ps.y << 64) | ps.x;
            mn = fminf(mn, mm.x);
            mx = fmaxf(mx, mm.y);
        }
    }
    const double sd = fx_to_double(sum);
    const float mean = __double2float_rn(__ddiv_rn(sd, (double)count));
    a.sum[k] = sd;
    a.vmin[k] = __float_as_uint(mn);
    a.vmax[k] = __float_as_uint(mx);
    a.mean[k] = mean;
    a.y[k] = a.tf[m * a.T + tf_entry(mean, (float)a.T, a.T - 1)];
    if (m == 0) a.count[p] = count;
}

// All fields of pixel p by one thread (the batched queries, which have many
// pixels over all pairs).
template <int M>
__device__ __forceinline__ void pixels_one(const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v,
                                           uint32_t p)
{
#pragma unroll 1
    for (int m = 0; m < M; ++m) pixels_field<M>(a, qa, v, p, m);
}

// One thread per (pixel, field): a pixel's fields are independent chains of
// table loads, run side by side (grid.y = field).
template <int M>
__global__ __launch_bounds__(256) void k_pixels(UpdateArgs a, QueryArgs qa, ValueTableArgs v)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.W) return;
    pixels_field<M>(a, qa, v, p, (int)blockIdx.y);
}

// The arguments of pair y of a batch: one TF's scan, one viewport's bins.
__device__ __forceinline__ void pair_args(const UpdateArgs& a, const BatchArgs& b, const PairDesc& pd,
                                          UpdateArgs& ak, QueryArgs& qk)
{
    ak = a;
    ak.W = pd.W;
    ak.tf = b.tfs + (uint64_t)pd.k * a.M * a.T;
    ak.sum = b.sum + pd.bin_off;
    ak.vmin = b.vmin + pd.bin_off;
    ak.vmax = b.vmax + pd.bin_off;
    ak.mean = b.mean + pd.bin_off;
    ak.y = b.y + pd.bin_off;
    ak.count = b.count + pd.cnt_off;
    qk.consts = b.consts + pd.k;
    qk.chunk_prefix = b.chunk_prefix + (uint64_t)pd.k * b.n_chunks;
    qk.step_sums = b.step_sums + (uint64_t)pd.k * b.n_chunks * STEPS;
    qk.H = b.H + pd.src_hs_off;
    qk.S = b.S + pd.src_hs_off;
    qk.psum = b.psum + pd.src_hs_off * 2 * a.M;
    qk.pmm = b.pmm + pd.src_hs_off * 2 * a.M;
    qk.hstride = pd.hstride;
}

template <int M, int PM>
__global__ __launch_bounds__(256) void k_bounds_batch(UpdateArgs a, BatchArgs b)
{
    extern __shared__ float s_tf[];
    const PairDesc pd = b.pairs[blockIdx.y];
    if (pd.derived || blockIdx.x * (blockDim.x >> 5) + 1 >= pd.W) return;   // block-uniform
    UpdateArgs ak;
    QueryArgs qk;
    pair_args(a, b, pd, ak, qk);
    load_table<M>(s_tf, ak.tf, a.T);
    __syncthreads();
    const uint32_t j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) + 1;
    if (j >= pd.W) return;
    bounds_one<M, PM>(ak, qk, s_tf, j, threadIdx.x & 31);
}

template <int M>
__global__ __launch_bounds__(256) void k_pixels_batch(UpdateArgs a, BatchArgs b, ValueTableArgs v)
{
    const PairDesc pd = b.pairs[blockIdx.y];
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pd.W) return;
    UpdateArgs ak;
    QueryArgs qk;
    pair_args(a, b, pd, ak, qk);
    pixels_one<M>(ak, qk, v, p);
}

template <int M, int PM>
cudaError_t run_bins(cudaStream_t s, const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v)
{
    if (a.n == 0 || a.W == 0) return cudaSuccess;
    const size_t smem = (size_t)M * (a.T + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_bounds<M, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.W > 1) k_bounds<M, PM><<<(a.W - 1 + 7) / 8, 256, smem, s>>>(a, qa);
    k_pixels<M><<<dim3((a.W + 255) / 256, M), 256, 0, s>>>(a, qa, v);
    return cudaGetLastError();
}

template <int M>
cudaError_t run_bins_m(cudaStream_t s, const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v)
{
    return a.prm.P == 1.0f ? run_bins<M, POW_ONE>(s, a, qa, v) : run_bins<M, POW_GEN>(s, a, qa, v);
}

template <int M, int PM>
cudaError_t run_bins_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b, const ValueTableArgs& v)
{
    if (a.n == 0 || b.n_pairs == 0) return cudaSuccess;
    const size_t smem = (size_t)M * (a.T + 1) * sizeof(float);
    static std::atomic<size_t> set_bytes[MAX_DEVICES];
    cudaError_t e = smem_attr_once(k_bounds_batch<M, PM>, smem, set_bytes);
    if (e != cudaSuccess) return e;
    if (b.max_W > 1) k_bounds_batch<M, PM><<<dim3((b.max_W - 1 + 7) / 8, b.n_pairs), 256, smem, s>>>(a, b);
    k_pixels_batch<M><<<dim3((b.max_W + 255) / 256, b.n_pairs), 256, 0, s>>>(a, b, v);
    return cudaGetLastError();
}

template <int M>
cudaError_t run_bins_batch_m(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b, const ValueTableArgs& v)
{
    return a.prm.P == 1.0f ? run_bins_batch<M, POW_ONE>(s, a, b, v) : run_bins_batch<M, POW_GEN>(s, a, b, v);
}

template <int M>
cudaError_t run_tables(cudaStream_t s, const ValueTableArgs& v, uint64_t* tot_lo, uint64_t* tot_hi)
{
    if (v.n_steps == 0) return cudaSuccess;
    const uint64_t warps_blocks = (v.n_steps + 7) / 8;
    k_vt_steps<M><<<(unsigned)(warps_blocks < 148ull * 16 ? warps_blocks : 148ull * 16), 256, 0, s>>>(v);
    const uint32_t nb = (uint32_t)((v.n_steps + 1023) / 1024);
    k_vt_scan1<<<dim3(nb, M), 256, 0, s>>>(v, tot_lo, tot_hi);
    k_vt_scan2<<<M, 32, 0, s>>>(v, tot_lo, tot_hi, nb);
    k_vt_scan3<<<dim3(nb, M), 256, 0, s>>>(v, tot_lo, tot_hi);
    for (int l = 1; l < v.n_levels; ++l) {
        const uint64_t n = v.n_steps + 1 - (2ull << (l - 1));
        const uint64_t blocks = (n + 255) / 256;
        k_vt_level<<<dim3((unsigned)(blocks < 4096 ? blocks : 4096), M), 256, 0, s>>>(v, l);
    }
    return cudaGetLastError();
}

}  // namespace

#define DVL_DISPATCH_M2(fn, MM, ...)              \
    switch (MM) {                                 \
        case 1: return fn<1>(__VA_ARGS__);        \
        case 2: return fn<2>(__VA_ARGS__);        \
        case 3: return fn<3>(__VA_ARGS__);        \
        case 4: return fn<4>(__VA_ARGS__);        \
        case 5: return fn<5>(__VA_ARGS__);        \
        case 6: return fn<6>(__VA_ARGS__);        \
        case 7: return fn<7>(__VA_ARGS__);        \
        case 8: return fn<8>(__VA_ARGS__);        \
        default: return cudaErrorInvalidValue;    \
    }

cudaError_t launch_value_tables(cudaStream_t s, uint32_t M, const ValueTableArgs& v, uint64_t* tot_lo,
                                uint64_t* tot_hi)
{
    DVL_DISPATCH_M2(run_tables, M, s, v, tot_lo, tot_hi)
}

cudaError_t launch_bins(cudaStream_t s, const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v)
{
    DVL_DISPATCH_M2(run_bins_m, a.M, s, a, qa, v)
}

cudaError_t launch_bins_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b, const ValueTableArgs& v)
{
    DVL_DISPATCH_M2(run_bins_batch_m, a.M, s, a, b, v)
}

uint64_t value_table_levels(uint64_t n_steps, uint64_t* stride)
{
    uint64_t levels = 1;                      // sparse table: levels 0 .. floor(log2(n_steps))
    while ((2ull << (levels - 1)) <= n_steps) ++levels;
    *stride = n_steps * levels;
    return levels;
}

}  // namespace dvl
