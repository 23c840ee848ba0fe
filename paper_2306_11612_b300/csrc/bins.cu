// Per-pixel bins as range queries (paper Sec. 3.2).
//
// In curve order the cells that touch pixel p form one contiguous range
// [lo_p, hi_p] (both the first and the last pixel of a cell's span are
// non-decreasing in the cell index).  The value a cell contributes to the bins
// is its normalised field value t, which does not depend on the transfer
// function.  So, once per data set and TF domain, this file builds value
// tables -- per 128-cell step, the exact fixed-point sum of t and its min/max,
// kept as prefixes within blocks of 32 steps plus a prefix of the block sums
// and a min/max sparse table over power-of-two runs of blocks -- and each
// update then needs only:
//   k_bounds  for every pixel boundary j, H(j) = number of cells whose span
//             starts before the boundary's first position C(j), and whether
//             the last of them also reaches pixel j ("straddles"); found by a
//             32-way search over the scan's chunk prefixes and an exact
//             recomputation of the widths of the one step that contains it.
//             It also records the partial-step sums/min/max of the two pixels
//             that meet in that step;
//   k_pixels  for every pixel: count = hi - lo + 1, sums from the prefix
//             tables plus the two recorded partial steps, min/max from the
//             block prefix/suffix entries, two sparse-table entries and the
//             records, then mean and the alpha of the mean.
// Sums are exact integer sums of floor(t * 2^95), so the bins do not depend
// on any summation order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bulk.cuh"
#include "cell_math.cuh"
#include "dvl_internal.h"

namespace dvl {

namespace {

typedef unsigned __int128 u128;
constexpr int FX_BITS = 95;          // fixed-point fraction bits of t

// floor(t * 2^95) for 0 <= t <= 1 (t a float32): t = mant * 2^(ex-150), so the
// value is mant shifted left by sh = ex - 150 + 95 (mant < 2^24, sh <= 72).
// Without branches (the lanes' cells differ in magnitude): PTX shifts clamp
// amounts >= 64 (and negative amounts, read as unsigned) to 64, giving 0, so
// lo = mant << sh or mant >> -sh and hi = mant << (sh - 64) or
// mant >> (64 - sh) each take two shifts.  For a zero or subnormal t the
// exponent field is 0, sh = -55 and every shift gives 0 (the value is below 1).
__device__ __forceinline__ uint64_t shl_clamp(uint64_t x, uint32_t s)
{
    uint64_t r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
__device__ __forceinline__ uint64_t shr_clamp(uint64_t x, uint32_t s)
{
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
__device__ __forceinline__ u128 fx_of(float t)
{
    const uint32_t b = __float_as_uint(t);              // t >= +0: no sign bit
    const uint64_t mant = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = (int)(b >> 23) - 150 + FX_BITS;
    const uint64_t lo = shl_clamp(mant, (uint32_t)sh) | shr_clamp(mant, (uint32_t)-sh);
    const uint64_t hi = shl_clamp(mant, (uint32_t)(sh - 64)) | shr_clamp(mant, (uint32_t)(64 - sh));
    return ((u128)hi << 64) | lo;
}

// floor(t 2^95) for 0 <= t <= 1 as five limbs, with float adds only (the
// FMA pipe): z = t 2^95 is exact; adding C = 2^95 with round-toward-zero
// leaves in the sum's mantissa field floor(z / 2^72) (the sum lies in
// [2^95, 2^96], whose spacing is 2^72), and z minus that multiple of 2^72 is
// exact (the bits of z below 2^72).  Repeating with C = 2^72, 2^49, 2^26 peels
// 23 bits at a time; the rest (< 8) is floored against 2^23.  The limbs are
// returned as the bit patterns of the rounded sums: bits(r_k) - bits(C_k) =
// floor of that part, so sums of the raw bits lose nothing (wrapping u32
// arithmetic), and floor(t 2^95) = L0 2^72 + L1 2^49 + L2 2^26 + L3 2^3 + L4.
__device__ __forceinline__ constexpr uint32_t limb_c(int k)
{
    return k == 0 ? 0x6F000000u : k == 1 ? 0x63800000u : k == 2 ? 0x58000000u : k == 3 ? 0x4C800000u : 0x4B000000u;
}
__device__ __forceinline__ void fx_limb_bits(float t, uint32_t (&r)[5])
{
    const float z0 = __fmul_rn(t, 0x1p95f);
    const float r0 = __fadd_rz(z0, 0x1p95f);
    const float z1 = __fsub_rn(z0, __fsub_rn(r0, 0x1p95f));
    const float r1 = __fadd_rz(z1, 0x1p72f);
    const float z2 = __fsub_rn(z1, __fsub_rn(r1, 0x1p72f));
    const float r2 = __fadd_rz(z2, 0x1p49f);
    const float z3 = __fsub_rn(z2, __fsub_rn(r2, 0x1p49f));
    const float r3 = __fadd_rz(z3, 0x1p26f);
    const float z4 = __fsub_rn(z3, __fsub_rn(r3, 0x1p26f));
    const float r4 = __fadd_rz(z4, 0x1p23f);
    r[0] = __float_as_uint(r0); r[1] = __float_as_uint(r1); r[2] = __float_as_uint(r2);
    r[3] = __float_as_uint(r3); r[4] = __float_as_uint(r4);
}

// The first two limbs only, enough for t = 0 and for t >= 2^-23: then
// t 2^95 >= 2^72 carries its 24 significant bits at 2^49 and above, so the
// limbs L2..L4 are 0.
__device__ __forceinline__ void fx_limb_bits2(float t, uint32_t& r0b, uint32_t& r1b)
{
    const float z0 = __fmul_rn(t, 0x1p95f);
    const float r0 = __fadd_rz(z0, 0x1p95f);
    const float z1 = __fsub_rn(z0, __fsub_rn(r0, 0x1p95f));
    r0b = __float_as_uint(r0);
    r1b = __float_as_uint(__fadd_rz(z1, 0x1p72f));
}

// The third limb's bits alone (L0 and L1 as fx_limb_bits2 gives them), enough
// with the first two for t = 0 and for t >= 2^-46: then t 2^95 >= 2^49 carries
// its bits at 2^26 and above, so L3 and L4 are 0.
__device__ __forceinline__ uint32_t fx_limb_bits_2(float t)
{
    const float z0 = __fmul_rn(t, 0x1p95f);
    const float r0 = __fadd_rz(z0, 0x1p95f);
    const float z1 = __fsub_rn(z0, __fsub_rn(r0, 0x1p95f));
    const float r1 = __fadd_rz(z1, 0x1p72f);
    const float z2 = __fsub_rn(z1, __fsub_rn(r1, 0x1p72f));
    return __float_as_uint(__fadd_rz(z2, 0x1p49f));
}

// The sum of floor(t 2^95) over `count` cells from the limb-bit sums
// (each limb's sum stays below 2^32 for count <= 256).
__device__ __forceinline__ u128 fx_from_limbs(const uint32_t (&acc)[5], uint32_t count)
{
    uint32_t L[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) L[k] = acc[k] - count * limb_c(k);
    return ((u128)L[0] << 72) + ((u128)L[1] << 49) + ((u128)L[2] << 26) + ((u128)L[3] << 3) + (u128)L[4];
}

__device__ __forceinline__ double fx_to_double(u128 x)
{
    const double hi = (double)(uint64_t)(x >> 64), lo = (double)(uint64_t)x;
    return (hi * 18446744073709551616.0 + lo) * 0x1.0p-95;
}

// ---- value tables ------------------------------------------------------------

__device__ __forceinline__ u128 shfl_up_u128(u128 x, int o)
{
    const uint64_t lo = __shfl_up_sync(FULL, (unsigned long long)(uint64_t)x, o);
    const uint64_t hi = __shfl_up_sync(FULL, (unsigned long long)(uint64_t)(x >> 64), o);
    return ((u128)hi << 64) | lo;
}

// Lane k holds step s0 + k of field m (sum of floor(t 2^95), min, max; lanes
// >= nst the neutral values).  The lanes scan across the block's steps: the
// exclusive prefix of the sums, the inclusive prefix and suffix min/max; lane
// 31's inclusive values are the block's total and (min, max).  Every table
// row is written once, coalesced.
__device__ __forceinline__ void vt_block_rows(const ValueTableArgs& v, int m, uint64_t b, int nst, int lane,
                                              u128 my_sum, uint32_t my_mn, uint32_t my_mx)
{
    const uint64_t s0 = b * VT_BLOCK;
    u128 incl = my_sum;
    uint32_t pmn = my_mn, pmx = my_mx, smn = my_mn, smx = my_mx;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u128 y = shfl_up_u128(incl, o);
        const uint32_t a = __shfl_up_sync(FULL, pmn, o), bb = __shfl_up_sync(FULL, pmx, o);
        const uint32_t c = __shfl_down_sync(FULL, smn, o), d = __shfl_down_sync(FULL, smx, o);
        if (lane >= o) { incl += y; pmn = min(pmn, a); pmx = max(pmx, bb); }
        if (lane + o < 32) { smn = min(smn, c); smx = max(smx, d); }
    }
    const u128 excl = incl - my_sum;
    const uint64_t row = (uint64_t)m * v.n_steps, s = s0 + lane;
    if (lane <= nst && s <= v.n_steps)      // entry n_steps: the prefix at the data set's end
        v.loc[(uint64_t)m * (v.n_steps + 1) + s] =
            make_ulonglong2((unsigned long long)(uint64_t)excl, (unsigned long long)(uint64_t)(excl >> 64));
    if (lane < nst) {
        v.raw[row + s] = make_float2(__uint_as_float(my_mn), __uint_as_float(my_mx));
        v.pre[row + s] = make_float2(__uint_as_float(pmn), __uint_as_float(pmx));
        v.suf[row + s] = make_float2(__uint_as_float(smn), __uint_as_float(smx));
    }
    if (lane == 31) {
        // block total into blk (turned into the exclusive prefix by k_vt_seg_*),
        // block (min, max) into level 0 of the sparse table
        v.blk[(uint64_t)m * (v.n_blocks + 1) + b] =
            make_ulonglong2((unsigned long long)(uint64_t)incl, (unsigned long long)(uint64_t)(incl >> 64));
        v.bmm[(uint64_t)m * v.b_levels * v.n_blocks + b] = make_float2(__uint_as_float(pmn), __uint_as_float(pmx));
    }
}

// Field m of block b with fewer than 32 full steps (the data set's last
// block), by one warp: lane k reads step k's cells from global memory (a
// float4 at a time; the padded rows make the reads past the last cell safe,
// and those cells are skipped) and sums all five limbs.
template <int M>
__device__ __noinline__ void vt_last_block_field(const ValueTableArgs& v, uint64_t b, int m, int lane)
{
    const uint64_t s0 = b * VT_BLOCK;
    const int nst = v.n_steps - s0 < (uint64_t)VT_BLOCK ? (int)(v.n_steps - s0) : VT_BLOCK;
    const float lo = v.consts->lo[m], sc = v.consts->s[m];
    uint32_t acc[5] = {0u, 0u, 0u, 0u, 0u}, count = 0u, mn = 0x7F800000u, mx = 0u;
    if (lane < nst) {
        const uint64_t c0 = (s0 + lane) * STEP;
        const float4* p = reinterpret_cast<const float4*>(v.val + m * v.pitch + c0);
        for (int cb = 0; cb < STEP / 32; ++cb) {
            float4 x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = __ldg(p + cb * 8 + j);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint64_t i0 = c0 + (uint64_t)(cb * 8 + j) * 4;
                const float e[4] = {x[j].x, x[j].y, x[j].z, x[j].w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (i0 + q < v.n) {
                        const float t = norm_t(e[q], lo, sc);
                        if (v.ent) {
                            const uint32_t en = floor_small(__fmul_rn(t, (float)v.T));
                            v.ent[m * v.pitch + ent_pos(i0 + q)] = (uint8_t)(en < v.T - 1u ? en : v.T - 1u);
                        }
                        uint32_t r[5];
                        fx_limb_bits(t, r);
#pragma unroll
                        for (int z = 0; z < 5; ++z) acc[z] += r[z];
                        ++count;
                        mn = min(mn, __float_as_uint(t));
                        mx = max(mx, __float_as_uint(t));
                    }
            }
        }
    }
    vt_block_rows(v, m, b, nst, lane, fx_from_limbs(acc, count), mn, mx);
}

// Blocks [0, n_full) whose 32 steps are all full, transposed: lane k owns
// step k of its warp's block and walks that step's cells itself, so a step's
// sum, min and max need no cross-lane reductions.  The sums are kept as five
// 32-bit limb sums (fx_limb_bits), mostly from two limbs: a stage whose cells
// all have t = 0 or t >= 2^-23 needs only L0 and L1; otherwise the warp
// walks the stage again for L2 alone (all t = 0 or >= 2^-46) or all five.  The cells reach shared
// memory by bulk copies: a stage holds VQ cells of each of the block's 32
// steps for one field (lane k's copy brings row k), VS stages per warp are
// in flight, and a (block, field) takes STEP / VQ stages.  Lane k reads its
// row's float4s starting at column k, so the 8 lanes of a quarter warp hit
// distinct banks.  Blocks go to the warps round-robin; the grid's last warps
// (those with the fewest full blocks) also take a last, partial block, a
// field each (vt_last_block_field).  A wait that runs out
// (bounded polls) sets ERR_TIMEOUT; the warp then waits, again bounded, for
// its copies in flight and stops.
constexpr int VT_WARPS = 4;
constexpr uint32_t VT_WAIT_POLLS = 4096;       // polls of <= 1 ms

// the stages and their barriers, then per warp one stage's entries (VQ bytes
// of each of the 32 rows) on their way out
template <int VQ, int VS>
constexpr size_t vt_tx_smem() { return (size_t)VT_WARPS * VS * (VT_BLOCK * VQ * 4 + 8) + (size_t)VT_WARPS * VT_BLOCK * VQ; }

template <int M, int VQ, int VS, bool ENT = false>
__global__ __launch_bounds__(VT_WARPS * 32) void k_vt_tx(ValueTableArgs v, uint64_t n_full)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int PARTS = STEP / VQ, C4 = VQ / 4;
    constexpr uint32_t STAGE = VT_BLOCK * VQ * 4;
    static_assert(STEP % VQ == 0 && VQ >= 32 && (C4 & (C4 - 1)) == 0, "stage rows: a power of two of >= 8 float4s");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t ring_s = sbase + (uint32_t)warp * VS * STAGE;
    const uint32_t bar_s = sbase + (uint32_t)(VT_WARPS * VS * STAGE) + (uint32_t)warp * VS * 8u;
    const float4* ring = reinterpret_cast<const float4*>(smem + (size_t)warp * VS * STAGE);
    const uint64_t gw = (uint64_t)blockIdx.x * VT_WARPS + warp, nw = (uint64_t)gridDim.x * VT_WARPS;
    if (gw == 0 && lane < M && v.n_steps % VT_BLOCK == 0)     // the prefix entry at the end, in a block of its own
        v.loc[(uint64_t)lane * (v.n_steps + 1) + v.n_steps] = make_ulonglong2(0ull, 0ull);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < VS; ++k) mbar_init(bar_s + 8u * k, 1);
        mbar_init_fence();
    }
    __syncwarp();
    // items in order: (block, field, part), blocks gw, gw + nw, ...; the
    // issue cursor runs up to VS items ahead of the consume cursor
    struct Cursor {
        uint64_t b;
        uint32_t m, h;
    };
    auto next = [&](Cursor& c) {
        if (++c.h == PARTS) {
            c.h = 0;
            if (++c.m == M) { c.m = 0; c.b += nw; }
        }
    };
    auto issue = [&](const Cursor& c, int k) {
        const uint32_t bar = bar_s + 8u * k;
        proxy_fence_shared();            // the warp's reads of the stage before the copy's writes
        if (lane == 0) mbar_arrive_expect_tx(bar, STAGE);
        bulk_g2s(ring_s + k * STAGE + (uint32_t)lane * VQ * 4,
                 v.val + c.m * v.pitch + (c.b * VT_BLOCK + lane) * STEP + c.h * VQ, VQ * 4, bar);
    };
    Cursor ci{gw, 0, 0}, cc{gw, 0, 0};
    int in_flight = 0;
    for (int k = 0; k < VS && ci.b < n_full; ++k, ++in_flight) { issue(ci, k); next(ci); }
    int k = 0;
    uint32_t phase = 0;
    bool late = false;
    uint32_t acc[5] = {0u, 0u, 0u, 0u, 0u};
    uint32_t mn = 0x7F800000u, mx = 0u;
    float lo = 0.f, sc = 0.f;
    const float Tf = (float)v.T;
    const uint32_t Tm1 = v.T - 1u;
    for (; cc.b < n_full; next(cc)) {
        if (cc.h == 0) {
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[q] = 0u;
            mn = 0x7F800000u; mx = 0u;
            lo = __ldg(&v.consts->lo[cc.m]); sc = __ldg(&v.consts->s[cc.m]);
        }
        if (!__all_sync(FULL, mbar_wait(bar_s + 8u * k, phase, VT_WAIT_POLLS))) { late = true; break; }   // warp-uniform
        const float4* row = ring + (size_t)k * (STAGE / 16) + lane * C4;
        // ENT: the entries of the lane's VQ cells, min(floor(t T), T - 1) as
        // k_entries writes them, 4 cells to a u32, go to the warp's row
        // buffer in shared memory and from there to global memory in whole
        // 16-byte pieces (the rows' VQ-byte segments are contiguous)
        uint32_t* ebuf = reinterpret_cast<uint32_t*>(smem + (size_t)VT_WARPS * VS * (STAGE + 8)) +
                         (size_t)warp * (VT_BLOCK * VQ / 4);
        uint32_t* erow = ebuf + lane * (VQ / 4);
        // first pass: min, max and the two-limb sums, valid when every t of
        // the warp's stage is 0 or >= 2^-23 (t bits - 1 >= bits(2^-23) - 1,
        // unsigned); otherwise a second pass takes all five limbs
        uint32_t a0 = 0u, a1 = 0u, okmin = 0xFFFFFFFFu;
#pragma unroll
        for (int c = 0; c < C4; ++c) {
            const float4 x = row[(c + lane) & (C4 - 1)];
            const float t0 = norm_t(x.x, lo, sc), t1 = norm_t(x.y, lo, sc);
            const float t2 = norm_t(x.z, lo, sc), t3 = norm_t(x.w, lo, sc);
            const uint32_t b0 = __float_as_uint(t0), b1 = __float_as_uint(t1);
            const uint32_t b2 = __float_as_uint(t2), b3 = __float_as_uint(t3);
            uint32_t p0, q0, p1, q1, p2, q2, p3, q3;
            fx_limb_bits2(t0, p0, q0); fx_limb_bits2(t1, p1, q1);
            fx_limb_bits2(t2, p2, q2); fx_limb_bits2(t3, p3, q3);
            a0 += (p0 + p1) + (p2 + p3);
            a1 += (q0 + q1) + (q2 + q3);
            mn = min(min(mn, b0), min(min(b1, b2), b3));
            mx = max(max(mx, b0), max(max(b1, b2), b3));
            okmin = min(min(okmin, b0 - 1u), min(min(b1 - 1u, b2 - 1u), b3 - 1u));
            if (ENT) {
                const uint32_t e0 = min(floor_small(__fmul_rn(t0, Tf)), Tm1), e1 = min(floor_small(__fmul_rn(t1, Tf)), Tm1);
                const uint32_t e2 = min(floor_small(__fmul_rn(t2, Tf)), Tm1), e3 = min(floor_small(__fmul_rn(t3, Tf)), Tm1);
                erow[(c + lane) & (C4 - 1)] = e0 | e1 << 8 | e2 << 16 | e3 << 24;
            }
        }
        if (ENT) {
            __syncwarp();
            const uint4* eb4 = reinterpret_cast<const uint4*>(ebuf);
#pragma unroll
            for (int r4 = 0; r4 < VT_BLOCK * VQ / 16 / 32; ++r4) {
                const int q = r4 * 32 + lane, row = q / (VQ / 16), part = q % (VQ / 16);
                const uint64_t i16 = (uint64_t)(cc.b * VT_BLOCK + row) * STEP + cc.h * VQ + part * 16;   // 16 cells
                *reinterpret_cast<uint4*>(v.ent + cc.m * v.pitch + ent_pos(i16)) = eb4[q];
            }
            __syncwarp();                // the buffer is refilled at the next stage
        }
        if (__all_sync(FULL, okmin >= 0x33FFFFFFu)) {
            acc[0] += a0;
            acc[1] += a1;
#pragma unroll
            for (int q = 2; q < 5; ++q) acc[q] += (uint32_t)VQ * limb_c(q);    // zero limbs of VQ cells
        } else if (__all_sync(FULL, okmin >= 0x287FFFFFu)) {                   // t = 0 or t >= 2^-46
            acc[0] += a0;
            acc[1] += a1;
            uint32_t a2 = 0u;
#pragma unroll 4
            for (int c = 0; c < C4; ++c) {
                const float4 x = row[(c + lane) & (C4 - 1)];
                a2 += (fx_limb_bits_2(norm_t(x.x, lo, sc)) + fx_limb_bits_2(norm_t(x.y, lo, sc))) +
                      (fx_limb_bits_2(norm_t(x.z, lo, sc)) + fx_limb_bits_2(norm_t(x.w, lo, sc)));
            }
            acc[2] += a2;
#pragma unroll
            for (int q = 3; q < 5; ++q) acc[q] += (uint32_t)VQ * limb_c(q);
        } else {
#pragma unroll 4
            for (int c = 0; c < C4; ++c) {
                const float4 x = row[(c + lane) & (C4 - 1)];
                uint32_t r0[5], r1[5], r2[5], r3[5];
                fx_limb_bits(norm_t(x.x, lo, sc), r0); fx_limb_bits(norm_t(x.y, lo, sc), r1);
                fx_limb_bits(norm_t(x.z, lo, sc), r2); fx_limb_bits(norm_t(x.w, lo, sc), r3);
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[q] += (r0[q] + r1[q]) + (r2[q] + r3[q]);
            }
        }
        __syncwarp();                    // every lane has read the stage
        --in_flight;
        if (ci.b < n_full) { issue(ci, k); next(ci); ++in_flight; }
        if (++k == VS) { k = 0; phase ^= 1u; }
        if (cc.h == PARTS - 1) vt_block_rows(v, (int)cc.m, cc.b, VT_BLOCK, lane, fx_from_limbs(acc, STEP), mn, mx);
    }
    if (late) {
        // the copies in flight fill the stages from k on, in order: each is
        // waited for once more (bounded) before the warp stops
        for (; in_flight > 0; --in_flight) {
            mbar_wait(bar_s + 8u * k, phase, VT_WAIT_POLLS);
            if (++k == VS) { k = 0; phase ^= 1u; }
        }
        if (lane == 0) atomicOr(v.err, ERR_TIMEOUT);
        return;
    }
    if (n_full < v.n_blocks)          // the last block's fields go to the grid's last warps
        for (uint64_t m = nw - 1 - gw; m < (uint64_t)M; m += nw) vt_last_block_field<M>(v, n_full, (int)m, lane);
}

// The block totals become their exclusive prefix per field (entry n_blocks:
// the field's total), in three launches over segments of VT_SEG blocks:
// k_vt_seg_sum writes each segment's total, k_vt_seg_scan (one warp per
// field) turns those into exclusive prefixes, and k_vt_seg_apply rescans each
// segment from its prefix.  Thread t of a segment's CTA takes blocks
// [t VT_PER, (t + 1) VT_PER) of it.
constexpr int VT_SEG_THREADS = 256, VT_PER = 8, VT_SEG = VT_SEG_THREADS * VT_PER;

__device__ __forceinline__ u128 ld_u128(const ulonglong2* p)
{
    const ulonglong2 x = *p;
    return ((u128)x.y << 64) | x.x;
}
__device__ __forceinline__ void st_u128(ulonglong2* p, u128 x)
{
    *p = make_ulonglong2((unsigned long long)(uint64_t)x, (unsigned long long)(uint64_t)(x >> 64));
}

// Exclusive scan of one value per thread over a CTA of VT_SEG_THREADS
// threads (warp shuffles, then the warp totals through shared memory);
// *total receives the CTA's sum.
__device__ __forceinline__ u128 cta_excl_scan_u128(u128 x, u128* s_warp, u128* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u128 incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u128 y = shfl_up_u128(incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    u128 before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < VT_SEG_THREADS / 32; ++w) {
        if (w < warp) before += s_warp[w];
        all += s_warp[w];
    }
    *total = all;
    return before + incl - x;
}

__global__ __launch_bounds__(VT_SEG_THREADS) void k_vt_seg_sum(ValueTableArgs v, ulonglong2* seg)
{
    __shared__ u128 s_warp[VT_SEG_THREADS / 32];
    const uint32_t m = blockIdx.y;
    const ulonglong2* blk = v.blk + (uint64_t)m * (v.n_blocks + 1);
    const uint64_t b0 = (uint64_t)blockIdx.x * VT_SEG + (uint64_t)threadIdx.x * VT_PER;
    u128 t = 0;
#pragma unroll
    for (int j = 0; j < VT_PER; ++j)
        if (b0 + j < v.n_blocks) t += ld_u128(blk + b0 + j);
    u128 total;
    cta_excl_scan_u128(t, s_warp, &total);
    if (threadIdx.x == 0) st_u128(seg + (uint64_t)m * gridDim.x + blockIdx.x, total);
}

__global__ void k_vt_seg_scan(ulonglong2* seg, uint32_t n_seg)
{
    const int lane = threadIdx.x & 31;
    ulonglong2* p = seg + (uint64_t)blockIdx.x * n_seg;
    u128 carry = 0;
    for (uint32_t s0 = 0; s0 < n_seg; s0 += 32) {
        const uint32_t i = s0 + lane;
        const u128 x = i < n_seg ? ld_u128(p + i) : (u128)0;
        u128 incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u128 y = shfl_up_u128(incl, o);
            if (lane >= o) incl += y;
        }
        if (i < n_seg) st_u128(p + i, carry + incl - x);
        const uint64_t lo = __shfl_sync(FULL, (unsigned long long)(uint64_t)incl, 31);
        const uint64_t hi = __shfl_sync(FULL, (unsigned long long)(uint64_t)(incl >> 64), 31);
        carry += ((u128)hi << 64) | lo;
    }
}

__global__ __launch_bounds__(VT_SEG_THREADS) void k_vt_seg_apply(ValueTableArgs v, const ulonglong2* seg)
{
    __shared__ u128 s_warp[VT_SEG_THREADS / 32];
    const uint32_t m = blockIdx.y;
    ulonglong2* blk = v.blk + (uint64_t)m * (v.n_blocks + 1);
    const uint64_t b0 = (uint64_t)blockIdx.x * VT_SEG + (uint64_t)threadIdx.x * VT_PER;
    u128 x[VT_PER], t = 0;
#pragma unroll
    for (int j = 0; j < VT_PER; ++j) {
        x[j] = b0 + j < v.n_blocks ? ld_u128(blk + b0 + j) : (u128)0;
        t += x[j];
    }
    u128 total;
    u128 run = ld_u128(seg + (uint64_t)m * gridDim.x + blockIdx.x) + cta_excl_scan_u128(t, s_warp, &total);
#pragma unroll
    for (int j = 0; j < VT_PER; ++j) {
        if (b0 + j < v.n_blocks) st_u128(blk + b0 + j, run);
        run += x[j];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == VT_SEG_THREADS - 1) st_u128(blk + v.n_blocks, run);
}

// Levels l, l + 1 and l + 2 (those below b_levels) of the blocks' sparse
// table from level l - 1: entry i of level l + j covers blocks
// [i, i + 2^(l + j)), i.e. level l - 1 entries i + r 2^(l - 1) for
// r < 2^(j + 1) (entries whose run would pass the last block are never read).
__global__ void k_vt_levels3(ValueTableArgs v, int l)
{
    const uint32_t m = blockIdx.y;
    const uint64_t h = 1ull << (l - 1), nb = v.n_blocks;
    float2* t = v.bmm + (uint64_t)m * v.b_levels * nb;
    const float2* prev = t + (uint64_t)(l - 1) * nb;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i + 2 * h <= nb;
         i += (uint64_t)gridDim.x * blockDim.x) {
        float2 acc = prev[i];
        int r = 1;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (l + j >= v.b_levels || i + (2 * h << j) > nb) break;
            for (; r < (2 << j); ++r) {
                const float2 e = prev[i + r * h];
                acc = make_float2(fminf(acc.x, e.x), fmaxf(acc.y, e.y));
            }
            t[(uint64_t)(l + j) * nb + i] = acc;
        }
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
// With alpha sums (qa.apart), also the fixed-point alpha sums of the same two
// cell sets, the alpha of a cell from the CTA's shared tables s_tf (T + 1
// entries per field).
// tt[k][m]: the normalised values of the lane's 4 cells of the step (those
// past the data set's end are not used).
template <int M>
__device__ __forceinline__ void step_partials(const UpdateArgs& a, const QueryArgs& qa, uint32_t j, uint64_t stb,
                                              uint64_t ste, uint64_t H, uint64_t first, int lane, const float* s_tf,
                                              const float (&tt)[4][M])
{
    const uint64_t idx = stb + lane * 4;
    const float Tf = (float)a.T;
    const uint32_t T1 = a.T + 1;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        // the sums of floor(t 2^95) as five limb-bit sums (fx_limb_bits; float
        // adds on the FMA pipe, then one 32-bit redux per limb)
        uint32_t tl[5] = {0u, 0u, 0u, 0u, 0u}, hl[5] = {0u, 0u, 0u, 0u, 0u};
        unsigned long long ta = 0, ha = 0;
        uint32_t tmn = 0x7F800000u, tmx = 0u, hmn = 0x7F800000u, hmx = 0u;
        if (idx < ste) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t cell = idx + k;
                const float t = tt[k][m];
                const uint32_t tb = __float_as_uint(t);
                uint32_t r[5];
                fx_limb_bits(t, r);
                const uint32_t af = qa.apart ? alpha_fx(s_tf[m * T1 + floor_small(__fmul_rn(t, Tf))]) : 0u;
                if (cell < H) {
#pragma unroll
                    for (int z = 0; z < 5; ++z) tl[z] += r[z];
                    ta += af;
                    tmn = min(tmn, tb);
                    tmx = max(tmx, tb);
                }
                if (cell >= first && cell < ste) {
#pragma unroll
                    for (int z = 0; z < 5; ++z) hl[z] += r[z];
                    ha += af;
                    hmn = min(hmn, tb);
                    hmx = max(hmx, tb);
                }
            }
        }
#pragma unroll
        for (int z = 0; z < 5; ++z) {
            tl[z] = __reduce_add_sync(FULL, tl[z]);
            hl[z] = __reduce_add_sync(FULL, hl[z]);
        }
        const u128 ts = fx_from_limbs(tl, (uint32_t)(H - stb));      // cells [stb, H)
        const u128 hs = fx_from_limbs(hl, (uint32_t)(ste - first));  // cells [first, ste)
        tmn = __reduce_min_sync(FULL, tmn);
        tmx = __reduce_max_sync(FULL, tmx);
        hmn = __reduce_min_sync(FULL, hmn);
        hmx = __reduce_max_sync(FULL, hmx);
        if (qa.apart) {                                            // uniform over the launch
            ta = warp_total_small(ta);
            ha = warp_total_small(ha);
        }
        if (lane == 0) {
            const uint64_t kt = ((uint64_t)j * 2 + 0) * M + m, kh = kt + M;
            qa.psum[kt] = make_ulonglong2((unsigned long long)(uint64_t)ts, (unsigned long long)(uint64_t)(ts >> 64));
            qa.pmm[kt] = make_float2(__uint_as_float(tmn), __uint_as_float(tmx));
            qa.psum[kh] = make_ulonglong2((unsigned long long)(uint64_t)hs, (unsigned long long)(uint64_t)(hs >> 64));
            qa.pmm[kh] = make_float2(__uint_as_float(hmn), __uint_as_float(hmx));
            if (qa.apart) {
                qa.apart[kt] = ta;
                qa.apart[kh] = ha;
            }
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
    float tt[4][M];                                       // the normalised values of the lane's cells
    if (C->linear) {                                      // widths 1: E_c = c
        H = X < a.n ? X : a.n;
        S = H >= 1 && (u128)H * a.W > jF;
        const uint64_t idx = (H - 1) / STEP * STEP + lane * 4;
        if (H >= 1 && idx < a.n) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(a.val + m * a.pitch + idx));
                tt[0][m] = norm_t(x.x, C->lo[m], C->s[m]);
                tt[1][m] = norm_t(x.y, C->lo[m], C->s[m]);
                tt[2][m] = norm_t(x.z, C->lo[m], C->s[m]);
                tt[3][m] = norm_t(x.w, C->lo[m], C->s[m]);
            }
        }
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
#pragma unroll
                for (int m = 0; m < M; ++m) tt[c][m] = norm_t(v[c][m], cc.lo[m], cc.s[m]);
                if (idx + c < a.n) q[c] = cc.width(tt[c], (L4 >> (8 * c)) & 0xFF, s_tf);
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
    step_partials<M>(a, qa, j, stb, ste, H, S ? H - 1 : H, lane, s_tf, tt);
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

// Prefix of the step sums of field m up to step s (steps [0, s)).
__device__ __forceinline__ u128 steps_prefix(const ValueTableArgs& v, uint32_t m, uint64_t s)
{
    const ulonglong2 a = v.blk[(uint64_t)m * (v.n_blocks + 1) + s / VT_BLOCK];
    const ulonglong2 b = v.loc[(uint64_t)m * (v.n_steps + 1) + s];
    return (((u128)a.y << 64) | a.x) + (((u128)b.y << 64) | b.x);
}

// Min/max of t over steps [s0, s1) (s0 < s1) of one field: inside one block
// the steps' own entries; across blocks the suffix of the first block, the
// prefix of the last one and, between them, two overlapping power-of-two
// runs of the blocks' sparse table.
__device__ __forceinline__ void steps_minmax(const ValueTableArgs& v, uint32_t m, uint64_t s0, uint64_t s1,
                                             float& mn, float& mx)
{
    const uint64_t row = (uint64_t)m * v.n_steps;
    const uint64_t b0 = s0 / VT_BLOCK, b1 = (s1 - 1) / VT_BLOCK;
    if (b0 == b1) {
        for (uint64_t s = s0; s < s1; ++s) {
            const float2 r = v.raw[row + s];
            mn = fminf(mn, r.x);
            mx = fmaxf(mx, r.y);
        }
        return;
    }
    const float2 a = v.suf[row + s0], b = v.pre[row + s1 - 1];
    mn = fminf(mn, fminf(a.x, b.x));
    mx = fmaxf(mx, fmaxf(a.y, b.y));
    if (b1 > b0 + 1) {
        const uint64_t c0 = b0 + 1, c1 = b1;                   // whole blocks [c0, c1)
        const int k = 63 - __clzll((long long)(c1 - c0));
        const float2* t = v.bmm + ((uint64_t)m * v.b_levels + (uint64_t)k) * v.n_blocks;
        const float2 x = t[c0], y = t[c1 - (1ull << k)];
        mn = fminf(mn, fminf(x.x, y.x));
        mx = fmaxf(mx, fmaxf(x.y, y.y));
    }
}

// Prefix of the fixed-point alpha sums of field m over steps [0, s): the
// exclusive prefix of s's chunk plus that of s within its chunk (s may be the
// step count, which ends a chunk when it is a multiple of STEPS).
__device__ __forceinline__ unsigned long long alpha_prefix(const QueryArgs& qa, uint32_t m, uint64_t s)
{
    const uint64_t c = s / STEPS, r = s - c * STEPS;
    const unsigned long long x = qa.achunk[(uint64_t)m * (qa.a_chunks + 1) + c];
    return r ? x + qa.astep[(uint64_t)m * qa.a_chunks * STEPS + s] : x;
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
        if (qa.apart) {
            a.asum[k] = 0.0;
            a.amean[k] = 0.0f;
        }
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
    unsigned long long asum = 0;                                     // fixed-point alpha sum
    if (one_step) {
        const float lo = C->lo[m], sc = C->s[m];
        for (uint64_t c = lo_c; c < c1; ++c) {
            const float t = norm_t(__ldg(a.val + m * a.pitch + c), lo, sc);
            sum += fx_of(t);
            mn = fminf(mn, t);
            mx = fmaxf(mx, t);
            if (qa.apart) {
                const uint32_t e = floor_small(__fmul_rn(t, (float)a.T));
                asum += alpha_fx(a.tf[m * a.T + (e < a.T ? e : a.T - 1)]);
            }
        }
    } else {
        if (qa.apart) {
            if (w1 > w0) asum = alpha_prefix(qa, m, w1) - alpha_prefix(qa, m, w0);
            if (has_l) asum += qa.apart[(bl * 2 + 1) * M + m];
            if (has_r) asum += qa.apart[(br * 2 + 0) * M + m];
        }
        if (w1 > w0) {
            steps_minmax(v, m, w0, w1, mn, mx);
            sum = steps_prefix(v, m, w1) - steps_prefix(v, m, w0);
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
    if (qa.apart) {
        const double as = (double)asum * (1.0 / 536870912.0);            // 2^-29; one rounding to double
        a.asum[k] = as;
        a.amean[k] = __double2float_rn(__ddiv_rn(as, (double)count));
    }
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
    qk.astep = nullptr;                      // batches have no alpha means
    qk.achunk = nullptr;
    qk.apart = nullptr;
    qk.a_chunks = 0;
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
    if (p < pd.W) {
        UpdateArgs ak;
        QueryArgs qk;
        pair_args(a, b, pd, ak, qk);
        pixels_one<M>(ak, qk, v, p);
    }
    if (b.stamps && blockIdx.x * blockDim.x < pd.W) {      // blocks with pixels: when they end
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(&b.stamps[1], global_ns());
    }
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

constexpr int VT_Q = 64, VT_S = 2;          // cells per stage row, stages per warp

template <int M>
cudaError_t run_tables(cudaStream_t s, const ValueTableArgs& v)
{
    if (v.n_blocks == 0) return cudaSuccess;
    const uint64_t n_full = v.n / ((uint64_t)VT_BLOCK * STEP);     // blocks of 32 full steps
    {
        const int ve = v.ent ? 1 : 0;                              // with the entries or without
        auto kernel = ve ? k_vt_tx<M, VT_Q, VT_S, true> : k_vt_tx<M, VT_Q, VT_S>;
        constexpr size_t smem = vt_tx_smem<VT_Q, VT_S>();
        static std::atomic<size_t> set_bytes[2][MAX_DEVICES];
        cudaError_t e = smem_attr_once(kernel, smem, set_bytes[ve]);
        int dev = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        // resident CTAs of the device, cached per thread for the last device
        thread_local int last_dev[2] = {-1, -1};
        thread_local uint64_t resident[2] = {0, 0};
        if (dev != last_dev[ve]) {
            int per_sm = 0, sms = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, VT_WARPS * 32, smem)) != cudaSuccess ||
                (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return e;
            resident[ve] = (uint64_t)(per_sm > 0 ? per_sm : 1) * sms;
            last_dev[ve] = dev;
        }
        const uint64_t need = (n_full + VT_WARPS - 1) / VT_WARPS;
        const uint64_t grid = need < resident[ve] ? (need ? need : 1) : resident[ve];
        kernel<<<(unsigned)grid, VT_WARPS * 32, smem, s>>>(v, n_full);
    }
    const uint32_t n_seg = (uint32_t)((v.n_blocks + VT_SEG - 1) / VT_SEG);
    k_vt_seg_sum<<<dim3(n_seg, M), VT_SEG_THREADS, 0, s>>>(v, v.seg);
    k_vt_seg_scan<<<M, 32, 0, s>>>(v.seg, n_seg);
    k_vt_seg_apply<<<dim3(n_seg, M), VT_SEG_THREADS, 0, s>>>(v, v.seg);
    for (int l = 1; l < v.b_levels; l += 3) {
        const uint64_t n = v.n_blocks + 1 - (2ull << (l - 1));
        const uint64_t blocks = (n + 255) / 256;
        k_vt_levels3<<<dim3((unsigned)(blocks < 1024 ? blocks : 1024), M), 256, 0, s>>>(v, l);
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

template <int M>
cudaError_t preload_bins_m()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)k_vt_tx<M, VT_Q, VT_S>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_vt_tx<M, VT_Q, VT_S, true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_vt_seg_sum);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_vt_seg_scan);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_vt_seg_apply);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_vt_levels3);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_bounds<M, POW_ONE>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void*)k_pixels<M>);
    return e;
}

cudaError_t preload_bins_kernels(uint32_t M)
{
    DVL_DISPATCH_M2(preload_bins_m, M)
}

cudaError_t launch_value_tables(cudaStream_t s, uint32_t M, const ValueTableArgs& v)
{
    DVL_DISPATCH_M2(run_tables, M, s, v)
}

cudaError_t launch_bins(cudaStream_t s, const UpdateArgs& a, const QueryArgs& qa, const ValueTableArgs& v)
{
    DVL_DISPATCH_M2(run_bins_m, a.M, s, a, qa, v)
}

cudaError_t launch_bins_batch(cudaStream_t s, const UpdateArgs& a, const BatchArgs& b, const ValueTableArgs& v)
{
    DVL_DISPATCH_M2(run_bins_batch_m, a.M, s, a, b, v)
}

uint64_t value_table_segments(uint64_t n_blocks)
{
    return (n_blocks + VT_SEG - 1) / VT_SEG;
}

int value_table_levels(uint64_t n_blocks)
{
    int levels = 0;                           // sparse table: levels 0 .. floor(log2(n_blocks))
    while (n_blocks >> levels) ++levels;
    return levels;
}

}  // namespace dvl
