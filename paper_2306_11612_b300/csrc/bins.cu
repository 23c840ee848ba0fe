// Per-pixel bins as range queries (paper Sec. 3.2).
//
// In curve order the cells that touch pixel p form one contiguous range
// [lo_p, hi_p] (both the first and the last pixel of a cell's span are
// non-decreasing in the cell index).  The value a cell contributes to the bins
// is its normalised field value t, which does not depend on the transfer
// function.  So, once per data set and TF domain, this file builds value
// tables -- per 128-cell step, the exact fixed-point sum of t and its min/max
// (plus an exclusive prefix of the sums and a base-16 min/max hierarchy) --
// and each update then needs only:
//   k_bounds  for every pixel boundary j, H(j) = number of cells whose span
//             starts before the boundary's first position C(j), and whether
//             the last of them also reaches pixel j ("straddles"); found by a
//             binary search over the scan's chunk prefixes and an exact
//             recomputation of the widths of the one step that contains it;
//   k_pixels  for every pixel: count = hi - lo + 1, sums from the prefix
//             table (with the partial steps at both ends added cell by cell),
//             min/max from the hierarchy, then mean and the alpha of the mean.
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

// floor(t * 2^95) for 0 <= t <= 1 (t a float32)
__device__ __forceinline__ u128 fx_of(float t)
{
    const uint32_t b = __float_as_uint(t);
    const uint32_t ex = (b >> 23) & 0xFF;
    if (ex == 0) return 0;                            // zero or subnormal: below 2^-126
    const uint64_t mant = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = (int)ex - 150 + FX_BITS;           // t = mant * 2^(ex-150)
    if (sh >= 0) return (u128)mant << sh;
    return sh > -24 ? (u128)(mant >> -sh) : (u128)0;
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

// Level l of the min/max hierarchy: entry i covers entries 16i..16i+15 of
// level l-1.
__global__ void k_vt_level(ValueTableArgs v, uint64_t off_prev, uint64_t n_prev, uint64_t off, uint64_t n)
{
    const uint32_t m = blockIdx.y;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float mn = 3.0f, mx = -1.0f;
        for (uint64_t c = 16 * i; c < 16 * i + 16 && c < n_prev; ++c) {
            mn = fminf(mn, v.mn[(uint64_t)m * v.level_stride + off_prev + c]);
            mx = fmaxf(mx, v.mx[(uint64_t)m * v.level_stride + off_prev + c]);
        }
        v.mn[(uint64_t)m * v.level_stride + off + i] = mn;
        v.mx[(uint64_t)m * v.level_stride + off + i] = mx;
    }
}

// ---- queries -------------------------------------------------------------------

// Pixel boundary j in [1, W-1]: H = #cells with span start E < C(j), and
// whether the last of them (cell H-1) has a positive width reaching past the
// real boundary j F / W (then it also touches pixel j).
template <int M, int PM>
__device__ __forceinline__ void bounds_one(const UpdateArgs& a, const QueryArgs& qa, const float* s_tf, uint32_t j,
                                           int lane)
{
    const UpdateConsts* C = qa.consts;
    const unsigned long long F = C->F;
    const PixelMap pm{F / a.W, F % a.W, F, a.W};
    const unsigned long long X = pm.C(j);
    const u128 jF = (u128)j * F;
    if (C->linear) {                                      // widths 1: E_c = c
        const unsigned long long H = X < a.n ? X : a.n;
        if (lane == 0) {
            qa.H[j] = H;
            qa.S[j] = H >= 1 && (u128)H * a.W > jF;
        }
        return;
    }
    // last chunk whose first cell starts before X (chunk 0 starts at 0 < X)
    const uint64_t n_chunks = (a.n + CHUNK - 1) / CHUNK;
    uint64_t lo = 0, hi = n_chunks - 1;
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) >> 1;
        if (qa.chunk_prefix[mid] < X) lo = mid; else hi = mid - 1;
    }
    const uint64_t chunk = lo, base = chunk * CHUNK;
    const uint64_t rem = a.n - base;
    const int nsteps = rem >= (uint64_t)CHUNK ? STEPS : (int)((rem + STEP - 1) / STEP);
    unsigned long long ssum = lane < nsteps ? qa.step_sums[chunk * STEPS + lane] : 0ull;
    const unsigned long long start = qa.chunk_prefix[chunk] + warp_incl_scan_u64(ssum, lane) - ssum;
    const unsigned before = __ballot_sync(FULL, lane < nsteps && start < X);
    const int st = 31 - __clz(before);                     // last step starting before X
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
    const int owner = 31 - __clz(has);                     // lane holding cell H-1
    const unsigned long long I = __shfl_sync(FULL, lastI, owner);
    const bool pos = __shfl_sync(FULL, lastpos, owner);
    if (lane == 0) {
        qa.H[j] = base + st * STEP + total;
        qa.S[j] = pos && (u128)I * a.W > jF;
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

// Range min/max of t over steps [s0, s1) of one field through the hierarchy.
__device__ __forceinline__ void steps_minmax(const ValueTableArgs& v, uint32_t m, uint64_t s0, uint64_t s1, int lane,
                                             float& mn, float& mx)
{
    uint64_t off = 0, n = v.n_steps;
    int l = 0;
    while (s0 < s1) {
        const float* bmn = v.mn + (uint64_t)m * v.level_stride + off;
        const float* bmx = v.mx + (uint64_t)m * v.level_stride + off;
        if (s1 - s0 <= 32 || l == v.n_levels - 1) {
            for (uint64_t k = s0 + lane; k < s1; k += 32) { mn = fminf(mn, bmn[k]); mx = fmaxf(mx, bmx[k]); }
            break;
        }
        const uint64_t a = (s0 + 15) & ~15ull, b = s1 & ~15ull;
        if (a >= b) {                                   // no whole parent block inside
            for (uint64_t k = s0 + lane; k < s1; k += 32) { mn = fminf(mn, bmn[k]); mx = fmaxf(mx, bmx[k]); }
            break;
        }
        if (lane < (int)(a - s0)) { mn = fminf(mn, bmn[s0 + lane]); mx = fmaxf(mx, bmx[s0 + lane]); }
        if (lane < (int)(s1 - b)) { mn = fminf(mn, bmn[b + lane]); mx = fmaxf(mx, bmx[b + lane]); }
        off += n;
        n = (n + 15) / 16;
        s0 = a / 16;
        s1 = b / 16;
        ++l;
    }
}

// Sum (fixed point), min and max of t over cells [c0, c1) that lie in one step.
template <int M>
__device__ __forceinline__ void cells_partial(const UpdateArgs& a, const float* lo, const float* sc, uint64_t c0,
                                              uint64_t c1, int lane, u128* sum, float* mn, float* mx)
{
    const uint64_t stb = c0 / STEP * STEP;
    const uint64_t idx = stb + lane * 4;
    if (c0 >= c1) return;
    if (idx + 3 < c0 || idx >= c1) return;
    const float* val = a.val;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(val + m * a.pitch + idx));
        const float c[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (idx + j >= c0 && idx + j < c1) {
                const float t = norm_t(c[j], lo[m], sc[m]);
                sum[m] += fx_of(t);
                mn[m] = fminf(mn[m], t);
                mx[m] = fmaxf(mx[m], t);
            }
    }
}

// One warp per pixel: the bins of cells [lo_p, hi_p].
template <int M>
__device__ __forceinline__ void pixels_one(const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v,
                                           uint32_t p, int lane)
{
    const uint64_t Hn = p + 1 < a.W ? qa.H[p + 1] : a.n;            // cells with E < C(p+1)
    const uint64_t lo_c = p == 0 ? 0 : (qa.S[p] ? qa.H[p] - 1 : qa.H[p]);
    const float Tf = (float)a.T;
    if (Hn == 0 || Hn - 1 < lo_c) {                                  // no cell touches p
        if (lane < M) {
            const uint64_t k = (uint64_t)lane * a.W + p;
            a.sum[k] = 0.0;
            a.vmin[k] = 0u;
            a.vmax[k] = 0u;
            a.mean[k] = 0.0f;
            a.y[k] = 0.0f;
        }
        if (lane == 0) a.count[p] = 0u;
        return;
    }
    const uint64_t hi_c = Hn - 1, c1 = hi_c + 1;
    const UpdateConsts* C = qa.consts;
    float lo[M], sc[M], mn[M], mx[M];
    u128 sum[M];
#pragma unroll
    for (int m = 0; m < M; ++m) { lo[m] = C->lo[m]; sc[m] = C->s[m]; mn[m] = 3.0f; mx[m] = -1.0f; sum[m] = 0; }
    const uint64_t s0 = lo_c / STEP, s1 = c1 / STEP;                 // steps of the two ends
    if (s0 == s1) {
        cells_partial<M>(a, lo, sc, lo_c, c1, lane, sum, mn, mx);
    } else {
        // head [lo_c, end of its step), tail [start of c1's step, c1)
        cells_partial<M>(a, lo, sc, lo_c, (s0 + 1) * STEP, lane, sum, mn, mx);
        cells_partial<M>(a, lo, sc, s1 * STEP, c1, lane, sum, mn, mx);
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        if (s1 > s0 + 1) steps_minmax(v, m, s0 + 1, s1, lane, mn[m], mx[m]);
        sum[m] = warp_sum_u128(sum[m]);
        mn[m] = warp_min(mn[m]);
        mx[m] = warp_max(mx[m]);
        if (s1 > s0 + 1) {                                            // whole steps from the prefix table
            const uint64_t row = (uint64_t)m * (v.n_steps + 1);
            const u128 pa = ((u128)v.pre_hi[row + s0 + 1] << 64) | v.pre_lo[row + s0 + 1];
            const u128 pb = ((u128)v.pre_hi[row + s1] << 64) | v.pre_lo[row + s1];
            sum[m] += pb - pa;
        }
    }
    const uint32_t count = (uint32_t)(c1 - lo_c);
    if (lane < M) {
        // each of the first M lanes writes one field (values are warp-uniform)
        double s = 0.0;
        float n_ = 0.0f, x_ = 0.0f;
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m == lane) { s = fx_to_double(sum[m]); n_ = mn[m]; x_ = mx[m]; }
        const uint64_t k = (uint64_t)lane * a.W + p;
        const float mean = __double2float_rn(__ddiv_rn(s, (double)count));
        a.sum[k] = s;
        a.vmin[k] = __float_as_uint(n_);
        a.vmax[k] = __float_as_uint(x_);
        a.mean[k] = mean;
        a.y[k] = a.tf[lane * a.T + tf_entry(mean, Tf, a.T - 1)];
    }
    if (lane == 0) a.count[p] = count;
}

template <int M>
__global__ __launch_bounds__(256) void k_pixels(UpdateArgs a, QueryArgs qa, ValueTableArgs v)
{
    const uint32_t p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= a.W) return;
    pixels_one<M>(a, qa, v, p, threadIdx.x & 31);
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
    qk.H = b.H + pd.hs_off;
    qk.S = b.S + pd.hs_off;
}

template <int M, int PM>
__global__ __launch_bounds__(256) void k_bounds_batch(UpdateArgs a, BatchArgs b)
{
    extern __shared__ float s_tf[];
    const PairDesc pd = b.pairs[blockIdx.y];
    if (blockIdx.x * (blockDim.x >> 5) + 1 >= pd.W) return;          // block-uniform
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
    const uint32_t p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= pd.W) return;
    UpdateArgs ak;
    QueryArgs qk;
    pair_args(a, b, pd, ak, qk);
    pixels_one<M>(ak, qk, v, p, threadIdx.x & 31);
}

template <int M, int PM>
cudaError_t run_bins(cudaStream_t s, const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v)
{
    if (a.n == 0 || a.W == 0) return cudaSuccess;
    const size_t smem = (size_t)M * (a.T + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_bounds<M, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.W > 1) k_bounds<M, PM><<<(a.W - 1 + 7) / 8, 256, smem, s>>>(a, qa);
    k_pixels<M><<<(a.W + 7) / 8, 256, 0, s>>>(a, qa, v);
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
    static size_t set_bytes = 0;                 // attribute set once per size (not during capture)
    if (smem > set_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_bounds_batch<M, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        set_bytes = smem;
    }
    if (b.max_W > 1) k_bounds_batch<M, PM><<<dim3((b.max_W - 1 + 7) / 8, b.n_pairs), 256, smem, s>>>(a, b);
    k_pixels_batch<M><<<dim3((b.max_W + 7) / 8, b.n_pairs), 256, 0, s>>>(a, b, v);
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
    uint64_t off_prev = 0, n_prev = v.n_steps, off = v.n_steps;
    for (int l = 1; l < v.n_levels; ++l) {
        const uint64_t n = (n_prev + 15) / 16;
        const uint64_t blocks = (n + 255) / 256;
        k_vt_level<<<dim3((unsigned)(blocks < 4096 ? blocks : 4096), M), 256, 0, s>>>(v, off_prev, n_prev, off, n);
        off_prev = off;
        off += n;
        n_prev = n;
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
    uint64_t n = n_steps, total = n_steps, levels = 1;
    while (n > 32) {
        n = (n + 15) / 16;
        total += n;
        ++levels;
    }
    *stride = total;
    return levels;
}

}  // namespace dvl
