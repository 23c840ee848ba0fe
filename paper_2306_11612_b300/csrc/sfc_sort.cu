// Once-per-data-set stage: input validation, per-field data ranges,
// space-filling-curve keys of every AMR cell, a stable LSD radix sort of the
// keys (single-pass "onesweep" digit scatter with decoupled look-back), and
// the gather of fields and levels into curve order.
//
// Paper: cells are a lower corner on the logical grid plus a level (Sec. 2.1);
// DVLs order cells by a space-filling-curve code of their quantised centroid
// (Sec. 2.2); the order is computed once and never changes (Sec. 4).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dvl_internal.h"
#include "logscale.cuh"

namespace dvl {

// ---- small device helpers --------------------------------------------------

__device__ __forceinline__ uint32_t float_to_ordered(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- validation and data ranges --------------------------------------------

__global__ void k_validate(uint64_t n, const int32_t* __restrict__ lower, size_t pitch,
                           const uint8_t* __restrict__ level, DataMeta* meta, uint32_t* err)
{
    uint32_t bad = 0, lmax = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t L = level[i];
        lmax = max(lmax, L);
        if (L > DVL_MAX_LEVEL) { bad |= ERR_LEVEL; continue; }
        int64_t w = 1ll << L;
        for (int d = 0; d < 3; ++d) {
            int64_t lo = lower[d * pitch + i];
            if (lo < 0 || lo + w > (1ll << DVL_MAX_LEVEL)) bad |= ERR_COORD;
        }
    }
    for (int o = 16; o; o >>= 1) {
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(err, bad);
        atomicMax(&meta->max_level, lmax);
    }
}

__global__ void k_field_ranges(uint64_t n, uint32_t M, const float* __restrict__ f, size_t pitch,
                               DataMeta* meta, uint32_t* err, bool positive)
{
    uint32_t m = blockIdx.y;
    const float* v = f + m * pitch;
    uint32_t mn = 0xFFFFFFFFu, mx = 0u, pos = 0xFFFFFFFFu, bad = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        float x = v[i];
        if (!isfinite(x)) { bad = ERR_NONFINITE; continue; }
        uint32_t o = float_to_ordered(x);
        mn = min(mn, o);
        mx = max(mx, o);
        if (x > 0.0f) pos = min(pos, __float_as_uint(x));   // positive floats order as their bits
    }
    for (int o = 16; o; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        pos = min(pos, __shfl_xor_sync(0xffffffffu, pos, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&meta->dmin[m], mn);
        atomicMax(&meta->dmax[m], mx);
        if (positive && pos != 0xFFFFFFFFu) atomicMin(&meta->dpos[m], pos);
        if (bad) atomicOr(err, bad);
    }
}

static int grid_for(uint64_t n, int threads)
{
    uint64_t b = (n + threads - 1) / threads;
    if (b > 148ull * 16) b = 148ull * 16;
    return b ? (int)b : 1;
}

void launch_validate(cudaStream_t s, uint64_t n, const int32_t* lower, const uint8_t* level,
                     uint32_t, float* const*, size_t pitch, DataMeta* meta, uint32_t* err)
{
    if (!n) return;
    k_validate<<<grid_for(n, 256), 256, 0, s>>>(n, lower, pitch, level, meta, err);
}

void launch_field_ranges(cudaStream_t s, uint64_t n, uint32_t M, const float* fields, size_t pitch,
                         DataMeta* meta, uint32_t* err, bool positive)
{
    if (!n) return;
    dim3 grid((unsigned)grid_for(n, 256) / M + 1, M);
    k_field_ranges<<<grid, 256, 0, s>>>(n, M, fields, pitch, meta, err, positive);
}

// ---- space-filling-curve keys ----------------------------------------------

// Spreads the low 21 bits of x so that bit k lands on bit 3k.
__device__ __forceinline__ unsigned long long spread3(uint32_t v)
{
    unsigned long long x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Hilbert code of a point with 21-bit coordinates, following Skilling,
// "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004): from the
// coarsest bit plane down, each axis either reflects the lower bits of axis 0
// (its own bit set) or swaps its lower bits with axis 0's; then the axes are
// Gray-coded and a plane-wise correction flips the lower bits.  The three
// transposed words are interleaved with axis 0 as the most significant bit of
// every 3-bit group.
__device__ __forceinline__ unsigned long long hilbert_key(uint32_t x, uint32_t y, uint32_t z)
{
    uint32_t a[3] = {x, y, z};
#pragma unroll 1
    for (int b = 20; b >= 1; --b) {
        const uint32_t bit = 1u << b, low = bit - 1u;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const bool set = (a[d] & bit) != 0;
            const uint32_t swap = (a[0] ^ a[d]) & low;
            // set: a0 ^= low; clear: exchange the low bits of a0 and a_d
            a[0] ^= set ? low : swap;
            if (d) a[d] ^= set ? 0u : swap;
        }
    }
    a[1] ^= a[0];
    a[2] ^= a[1];
    uint32_t t = 0;
#pragma unroll 1
    for (int b = 20; b >= 1; --b)
        if (a[2] & (1u << b)) t ^= (1u << b) - 1u;
    a[0] ^= t;
    a[1] ^= t;
    a[2] ^= t;
    return (spread3(a[0]) << 2) | (spread3(a[1]) << 1) | spread3(a[2]);
}

__global__ void k_keys(uint64_t n, const int32_t* __restrict__ lower, size_t pitch,
                       const uint8_t* __restrict__ level, int sfc, unsigned long long* keys,
                       uint32_t* vals, uint32_t* hist, DataMeta* meta)
{
    __shared__ uint32_t s_hist[8 * RS_RADIX];
    for (int i = threadIdx.x; i < 8 * RS_RADIX; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    unsigned long long kor = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t w = 1u << level[i];
        uint32_t cx = 2u * (uint32_t)lower[i] + w;            // exact centroid,
        uint32_t cy = 2u * (uint32_t)lower[pitch + i] + w;    // half-cell units
        uint32_t cz = 2u * (uint32_t)lower[2 * pitch + i] + w;
        unsigned long long k = sfc == DVL_SFC_HILBERT
                                   ? hilbert_key(cx, cy, cz)
                                   : (spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2));
        keys[i] = k;
        vals[i] = (uint32_t)i;
        kor |= k;
#pragma unroll
        for (int d = 0; d < 8; ++d) atomicAdd(&s_hist[d * RS_RADIX + ((k >> (8 * d)) & 0xFF)], 1u);
    }
    for (int o = 16; o; o >>= 1) kor |= __shfl_xor_sync(0xffffffffu, kor, o);
    if ((threadIdx.x & 31) == 0 && kor) atomicOr(&meta->key_or, kor);
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * RS_RADIX; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

void launch_keys(cudaStream_t s, uint64_t n, const int32_t* lower, size_t pitch, const uint8_t* level,
                 int sfc, unsigned long long* keys, uint32_t* vals, uint32_t* hist, DataMeta* meta)
{
    if (!n) return;
    k_keys<<<grid_for(n, 256), 256, 0, s>>>(n, lower, pitch, level, sfc, keys, vals, hist, meta);
}

// ---- onesweep radix pass ---------------------------------------------------
// Status word: [63:40] epoch, [33:32] flag (1 = tile count, 2 = inclusive
// prefix over tiles), [31:0] value.  Words of other epochs read as "not yet".

__device__ __forceinline__ unsigned long long rs_pack(uint32_t epoch, uint32_t flag, uint32_t v)
{
    return ((unsigned long long)epoch << 40) | ((unsigned long long)flag << 32) | v;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t x, uint32_t* s_tmp /*8*/)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < warp; ++w) off += s_tmp[w];
    __syncthreads();
    return off + incl - x;
}

__global__ __launch_bounds__(RS_THREADS) void k_onesweep(
    uint32_t n, const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
    unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout, int shift,
    const uint32_t* __restrict__ hist_digit, unsigned long long* status, uint32_t epoch,
    uint32_t* tile_counter, uint32_t* err, long long spin_limit)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_keys = reinterpret_cast<unsigned long long*>(smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + RS_TILE);
    uint32_t* s_whist = s_vals + RS_TILE;                 // [8 warps][256]
    __shared__ uint32_t s_tileoff[RS_RADIX], s_gbase[RS_RADIX], s_tmp[8], s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < 8 * RS_RADIX; i += RS_THREADS) s_whist[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t base = (uint64_t)tile * RS_TILE;

    // 1. load (warp-contiguous runs) and rank within the warp, stably
    unsigned long long k[RS_KPT];
    uint32_t v[RS_KPT], rank[RS_KPT];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < RS_KPT; ++i) {
        uint64_t idx = base + (uint64_t)warp * (32 * RS_KPT) + i * 32 + lane;
        bool valid = idx < n;
        k[i] = valid ? kin[idx] : ~0ull;
        v[i] = valid ? vin[idx] : 0u;
        uint32_t d = valid ? (uint32_t)((k[i] >> shift) & 0xFF) : 0x100u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? s_whist[warp * RS_RADIX + d] : 0u;
        __syncwarp();
        if (valid && (peers & lt_mask) == 0) s_whist[warp * RS_RADIX + d] = before + __popc(peers);
        __syncwarp();
        rank[i] = before + __popc(peers & lt_mask);
    }
    __syncthreads();

    // 2. per digit (thread = digit): warp offsets, tile count
    const uint32_t d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t c = s_whist[w * RS_RADIX + d];
        s_whist[w * RS_RADIX + d] = run;
        run += c;
    }
    const uint32_t tile_cnt = run;

    // 3. decoupled look-back over tiles for this digit
    unsigned long long* my = status + (uint64_t)tile * RS_RADIX + d;
    uint32_t excl = 0;
    if (tile == 0) {
        st_relaxed(my, rs_pack(epoch, 2, tile_cnt));
    } else {
        st_relaxed(my, rs_pack(epoch, 1, tile_cnt));
        int64_t j = (int64_t)tile - 1;
        long long spins = 0;
        while (j >= 0) {
            unsigned long long w = ld_relaxed(status + (uint64_t)j * RS_RADIX + d);
            uint32_t flag = (uint32_t)(w >> 32) & 3u;
            if ((uint32_t)(w >> 40) != epoch || flag == 0) {
                if (++spins > spin_limit) { atomicOr(err, ERR_TIMEOUT); break; }
                __nanosleep(100);
                continue;
            }
            excl += (uint32_t)w;
            if (flag == 2) break;
            --j;
        }
        st_relaxed(my, rs_pack(epoch, 2, excl + tile_cnt));
    }
    uint32_t gstart = block_excl_scan256(hist_digit[d], s_tmp);
    uint32_t toff = block_excl_scan256(tile_cnt, s_tmp);
    s_gbase[d] = gstart + excl;
    s_tileoff[d] = toff;
    __syncthreads();

    // 4. place into shared memory in tile-sorted order
#pragma unroll
    for (int i = 0; i < RS_KPT; ++i) {
        uint64_t idx = base + (uint64_t)warp * (32 * RS_KPT) + i * 32 + lane;
        if (idx < n) {
            uint32_t dg = (uint32_t)((k[i] >> shift) & 0xFF);
            uint32_t lp = s_tileoff[dg] + s_whist[warp * RS_RADIX + dg] + rank[i];
            s_keys[lp] = k[i];
            s_vals[lp] = v[i];
        }
    }
    __syncthreads();

    // 5. coalesced write-out: consecutive threads write consecutive slots of a digit run
    const uint32_t tile_valid = (n - base) < (uint64_t)RS_TILE ? (uint32_t)(n - base) : (uint32_t)RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_KPT; ++i) {
        uint32_t idx = i * RS_THREADS + tid;
        if (idx < tile_valid) {
            unsigned long long key = s_keys[idx];
            uint32_t dg = (uint32_t)((key >> shift) & 0xFF);
            uint32_t dest = s_gbase[dg] + (idx - s_tileoff[dg]);
            if (dest < n) {          // only false after a timed-out wait
                kout[dest] = key;
                vout[dest] = s_vals[idx];
            }
        }
    }
}

cudaError_t launch_onesweep(cudaStream_t s, uint64_t n, const unsigned long long* kin,
                            const uint32_t* vin, unsigned long long* kout, uint32_t* vout, int shift,
                            const uint32_t* hist_digit, unsigned long long* status, uint32_t epoch,
                            uint32_t* tile_counter, uint32_t* err, int64_t spin_limit)
{
    if (!n) return cudaSuccess;
    const size_t smem = (size_t)RS_TILE * (8 + 4) + 8 * RS_RADIX * 4;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    unsigned tiles = (unsigned)((n + RS_TILE - 1) / RS_TILE);
    k_onesweep<<<tiles, RS_THREADS, smem, s>>>((uint32_t)n, kin, vin, kout, vout, shift, hist_digit,
                                               status, epoch, tile_counter, err, spin_limit);
    return cudaGetLastError();
}

// ---- gather into curve order ----------------------------------------------

__global__ void k_gather(uint64_t n, const uint32_t* __restrict__ perm, uint32_t M,
                         const float* __restrict__ fin, size_t pin, const uint8_t* __restrict__ lin,
                         float* __restrict__ fout, size_t pout, uint8_t* __restrict__ lout,
                         uint32_t log_mask, const DataMeta* __restrict__ meta)
{
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n;
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t i = perm[k];
        if (i >= n) continue;        // only after a failed sort (error already raised)
        if (lin) lout[k] = lin[i];
        for (uint32_t m = 0; m < M; ++m) {
            float x = fin[m * pin + i];
            if (log_mask >> m & 1u) x = log10_scale(x > 0.0f ? x : __uint_as_float(meta->dpos[m]));
            fout[m * pout + k] = x;
        }
    }
}

void launch_gather(cudaStream_t s, uint64_t n, const uint32_t* perm, uint32_t M, const float* fin,
                   size_t pitch_in, const uint8_t* lin, float* fout, size_t pitch_out, uint8_t* lout,
                   uint32_t log_mask, const DataMeta* meta)
{
    if (!n) return;
    k_gather<<<grid_for(n, 256), 256, 0, s>>>(n, perm, M, fin, pitch_in, lin, fout, pitch_out, lout,
                                              log_mask, meta);
}

}  // namespace dvl
