// Device-side building blocks shared by the update, adjoint and bin-query
// kernels: the per-cell arithmetic of the method (normalisation, TF entry,
// variation, importance, fixed-point width) and the exact pixel boundaries.
// Included by .cu files only; everything is internal to each translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dvl_internal.h"

namespace dvl {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long FLAG_A = 1ull << 62;   // tile aggregate published
constexpr unsigned long long FLAG_P = 2ull << 62;   // inclusive prefix published
constexpr unsigned long long VAL_MASK = (1ull << 62) - 1;

// exponent modes of the per-cell kernels: P == 1, or any other P (exact
// products/sqrt when 2P is an integer in [0, 16], powf otherwise)
enum { POW_ONE = 0, POW_GEN = 1 };

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

// The device's global nanosecond clock.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float ordered_to_float(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// 2^e as a float for -126 <= e <= 127 (exact).
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((127 + e) << 23); }

// Normalised value t = clamp((v - lo) * s, 0, 1) (Sec. 3.3).  The clamp works
// on the bit pattern: negative values and -0 become +0, values above 1 (and
// +inf) become 1.  NaN cannot occur: field values are finite (checked at
// load), lo is finite and s is finite (k_prepare sets lo = 0 where s = 0).
__device__ __forceinline__ float norm_t(float v, float lo, float s)
{
    int b = __float_as_int(__fmul_rn(__fsub_rn(v, lo), s));
    b = min(max(b, 0), 0x3F800000);
    return __int_as_float(b);
}

// TF entry of t: min(floor(t T), T - 1) (used by the non-hot kernels).
__device__ __forceinline__ uint32_t tf_entry(float t, float Tf, uint32_t Tm1)
{
    uint32_t a = (uint32_t)__fmul_rn(t, Tf);    // t*T >= 0: truncation == floor
    return a < Tm1 ? a : Tm1;
}

// floor(x) for 0 <= x < 2^23: adding 2^23 with round-toward-zero keeps the
// integer part in the low mantissa bits.
__device__ __forceinline__ uint32_t floor_small(float x)
{
    return __float_as_uint(__fadd_rz(x, 8388608.0f)) - 0x4B000000u;
}

// x^P with n2 = 2P for the exact modes (sqrt once if n2 is odd, then
// left-to-right products); n2 < 0 selects powf.
__device__ __forceinline__ float pow_gen(float x, int n2, float P)
{
    if (n2 < 0) return powf(x, P);
    if (n2 == 0) return 1.0f;
    float b;
    int k;
    if (n2 & 1) { b = __fsqrt_rn(x); k = n2; } else { b = x; k = n2 >> 1; }
    float y = b;
    for (int i = 1; i < k; ++i) y = __fmul_rn(y, b);
    return y;
}

// Eq. 3 with the minimum importance m.  Both placements in one branch-free
// form: before-scale f = (max(r, m) 2^L)^P, after-power f = max((r 2^L)^P, m);
// mb / ma hold m in the selected slot and 0 in the other (max with 0 is the
// identity here since r >= +0 and x^P >= +0).
template <int PM>
__device__ __forceinline__ float importance(float V, uint32_t L, float inv_vmax, float mb, float ma, int wshift,
                                            int n2, float P)
{
    float r = fmaxf(__fmul_rn(V, inv_vmax), mb);
    float x = __fmul_rn(r, exp2i((int)L * wshift));
    float f = PM == POW_ONE ? x : pow_gen(x, n2, P);
    return fmaxf(f, ma);
}

// Two float32 operations in one instruction (sm_100 and later; each half
// rounded on its own, exactly as the scalar form).
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mul.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 fma_rz2(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{\n\t.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mov.b64 c, {%6, %7};\n\tfma.rz.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// Three-input float max / min (single instructions on sm_100 and later); the
// result is one of the inputs, as with fmaxf / fminf on non-NaN values.
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// max_m al[m] and min_m al[m] (the ends of Eq. 1 for one cell), with
// three-input steps.
template <int M>
__device__ __forceinline__ void spread_ends(const float (&al)[M], float& hi_out, float& lw_out)
{
    float hi = al[0], lw = al[0];
    int m = 1;
#pragma unroll
    for (; m + 1 < M; m += 2) {
        hi = max3f(hi, al[m], al[m + 1]);
        lw = min3f(lw, al[m], al[m + 1]);
    }
    if (m < M) {
        hi = fmaxf(hi, al[m]);
        lw = fminf(lw, al[m]);
    }
    hi_out = hi;
    lw_out = lw;
}

// Eq. 1: max_m al[m] - min_m al[m].
template <int M>
__device__ __forceinline__ float spread(const float (&al)[M])
{
    float hi, lw;
    spread_ends<M>(al, hi, lw);
    return __fsub_rn(hi, lw);
}

// Fast TF entry for a power-of-two table size T (then t*T is exact):
//   t = clamp(fl((v - lo) * s), 0, 1)  one multiply with saturation (NaN -> 0;
//                                      the sign of a zero t does not matter here),
//   floor(t * T) + 2^23               one fma rounded toward zero,
// and the shared-memory address of the entry from that result's bits in one
// multiply-add: c_m = table address of field m - 4 * bits(2^23) (mod 2^32).
// The entry equals min(floor(t*T), T) of the general path bit for bit.
__device__ __forceinline__ float mul_sat(float a, float b)
{
    float r;
    asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float fma_rz(float a, float b, float c)
{
    float r;
    asm("fma.rz.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float r;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(addr));
    return r;
}
constexpr uint32_t BITS_2P23 = 0x4B000000u;         // bits of 2^23

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t r;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(addr));
    return r;
}

// A cell's alpha in the fixed point of the alpha-mean sums: rint(alpha 2^29)
// (alpha in [0, 1], so at most 2^29 and the 4 cells of a lane fit in 32 bits;
// the scaling is exact).  Every kernel that adds alphas converts with this one
// function, so the sums are exact integers and independent of the order of
// addition.
constexpr float ALPHA_FX_ONE = 536870912.0f;         // 2^29
__device__ __forceinline__ uint32_t alpha_fx(float A) { return __float2uint_rn(__fmul_rn(A, ALPHA_FX_ONE)); }

// Per-cell constants in registers, specialised on the field count M and the
// exponent mode.  The alpha tables live in shared memory with T+1 entries per
// field (entry T repeats entry T-1) so that t = 1 needs no clamp.
template <int M, int PM>
struct Cell {
    float lo[M], s[M];
    float inv_vmax, mb, ma, qscale, P, Tf;
    float ivq, mbq, maq;               // inv_vmax, mb and ma times 2^Q (see q2_pow1)
    int n2, wshift, T1;
    bool linear;

    __device__ __forceinline__ void load(const UpdateConsts* C, uint32_t T)
    {
#pragma unroll
        for (int m = 0; m < M; ++m) { lo[m] = C->lo[m]; s[m] = C->s[m]; }
        inv_vmax = C->inv_vmax;
        const bool after = C->min_imp_mode == DVL_MINIMP_AFTER_POWER;
        mb = after ? 0.0f : C->min_imp;
        ma = after ? C->min_imp : 0.0f;
        qscale = C->qscale;
        ivq = __fmul_rn(inv_vmax, qscale);
        mbq = __fmul_rn(mb, qscale);
        maq = __fmul_rn(ma, qscale);
        P = C->P;
        n2 = C->pow_n2;
        wshift = C->width_shift;
        Tf = (float)T;
        T1 = (int)T + 1;
        linear = C->linear != 0;
    }

    // Eq. 1 over the M fields of one cell, from normalised values t[].
    __device__ __forceinline__ float variation(const float* t, const float* s_tf) const
    {
        float al[M];
#pragma unroll
        for (int m = 0; m < M; ++m) al[m] = s_tf[m * T1 + floor_small(__fmul_rn(t[m], Tf))];
        return spread<M>(al);
    }

    // fixed-point width of a cell: rint(f 2^Q) (<= 2^31)
    __device__ __forceinline__ uint32_t width(const float* t, uint32_t L, const float* s_tf) const
    {
        float f = importance<PM>(variation(t, s_tf), L, inv_vmax, mb, ma, wshift, n2, P);
        return __float2uint_rn(__fmul_rn(f, qscale));
    }

    // the same width from the raw field values, T a power of two (see
    // mul_sat / fma_rz); cm[m] = shared address of field m's table - 4 bits(2^23)
    __device__ __forceinline__ uint32_t width_p2(const float* v, uint32_t L, const uint32_t* cm) const
    {
        float al[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float t = mul_sat(__fsub_rn(v[m], lo[m]), s[m]);
            al[m] = lds_f32(__float_as_uint(fma_rz(t, Tf, 8388608.0f)) * 4u + cm[m]);
        }
        float f = importance<PM>(spread<M>(al), L, inv_vmax, mb, ma, wshift, n2, P);
        return __float2uint_rn(__fmul_rn(f, qscale));
    }

    // Eq. 3 with P = 1 and the fixed-point width of two cells from the ends
    // of their spreads (ha - la, hb - lb) and their level factors Sa, Sb
    // (2^(L wshift)).  With qs = 2^Q,
    //   rint(max(max(fl(V inv), mb) S, ma) qs)
    //     = rint(max(fl(V fl(inv qs)) S, fl(mb qs) S, fl(ma qs))):
    // Q is chosen so that fu 2^Q <= 2^31, which keeps inv qs, mb qs and ma qs
    // finite and inv qs normal (inv >= 1); scaling by a power of two is exact
    // in the normal range, rounding is monotone (it commutes with max), and a
    // value that leaves the normal range lies far below 1/2 on both sides.
    // One 3-input max per cell instead of two maxima and a multiply.
    __device__ __forceinline__ void q2_pow1(float ha, float la, float hb, float lb, float Sa, float Sb,
                                            uint32_t& qa, uint32_t& qb) const
    {
        const float2 S = make_float2(Sa, Sb);
        const float2 V = sub2(make_float2(ha, hb), make_float2(la, lb));
        const float2 x = mul2(mul2(V, make_float2(ivq, ivq)), S);
        const float2 fl = mul2(make_float2(mbq, mbq), S);
        qa = __float2uint_rn(max3f(x.x, fl.x, maq));
        qb = __float2uint_rn(max3f(x.y, fl.y, maq));
    }

    // width_p2 of two cells a and b at once (P = 1): the subtraction, the
    // entry's fma and Eq. 3's multiplies in float32x2 form, bit for bit the
    // same as two width_p2 calls.  AL: also returns each field's fixed-point
    // alpha of the two cells in axa[m], axb[m] (see width_p2_alpha).
    template <bool AL>
    __device__ __forceinline__ void width2_p2(const float* va, const float* vb, uint32_t La, uint32_t Lb,
                                              const uint32_t* cm, uint32_t aoff, uint32_t (&axa)[M],
                                              uint32_t (&axb)[M], uint32_t& qa, uint32_t& qb) const
    {
        float ala[M], alb[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float2 d = sub2(make_float2(va[m], vb[m]), make_float2(lo[m], lo[m]));
            const float2 e = fma_rz2(make_float2(mul_sat(d.x, s[m]), mul_sat(d.y, s[m])), make_float2(Tf, Tf),
                                     make_float2(8388608.0f, 8388608.0f));
            const uint32_t adra = __float_as_uint(e.x) * 4u + cm[m], adrb = __float_as_uint(e.y) * 4u + cm[m];
            ala[m] = lds_f32(adra);
            alb[m] = lds_f32(adrb);
            if (AL) {
                axa[m] = lds_u32(adra + aoff);
                axb[m] = lds_u32(adrb + aoff);
            }
        }
        float ha, la, hb, lb;
        spread_ends<M>(ala, ha, la);
        spread_ends<M>(alb, hb, lb);
        q2_pow1(ha, la, hb, lb, exp2i((int)La * wshift), exp2i((int)Lb * wshift), qa, qb);
    }

    // The width from the cell's TF entries e[m] (precomputed for the TF
    // domain: min(floor(t T), T - 1), the entry every path above reads),
    // tb[m] = shared address of field m's table; the same value as width().
    __device__ __forceinline__ uint32_t width_ent(const uint32_t* e, uint32_t L, const uint32_t* tb) const
    {
        float al[M];
#pragma unroll
        for (int m = 0; m < M; ++m) al[m] = lds_f32(tb[m] + 4u * e[m]);
        float f = importance<PM>(spread<M>(al), L, inv_vmax, mb, ma, wshift, n2, P);
        return __float2uint_rn(__fmul_rn(f, qscale));
    }

    // width_ent of two cells at once (P = 1), Eq. 3's arithmetic in
    // float32x2 form as in width2_p2.  AL: also returns each field's
    // fixed-point alpha of the two cells (the u32 twin tables lie `aoff`
    // bytes after the float ones).
    template <bool AL>
    //   four = 4 and w23 = wshift << 23 are run-time values, so that the
    // table addresses (tb + 4 e) and the level factors (the bits of
    // 2^(L wshift) = L (wshift << 23) + bits(1)) are integer multiply-adds on
    // the FMA pipe rather than shifts and adds on the busier integer pipe.
    __device__ __forceinline__ void width2_ent(const uint32_t* ea, const uint32_t* eb, uint32_t La, uint32_t Lb,
                                               const uint32_t* tb, uint32_t aoff, uint32_t (&axa)[M],
                                               uint32_t (&axb)[M], uint32_t& qa, uint32_t& qb, uint32_t four,
                                               uint32_t w23) const
    {
        float ala[M], alb[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const uint32_t adra = ea[m] * four + tb[m], adrb = eb[m] * four + tb[m];
            ala[m] = lds_f32(adra);
            alb[m] = lds_f32(adrb);
            if (AL) {
                axa[m] = lds_u32(adra + aoff);
                axb[m] = lds_u32(adrb + aoff);
            }
        }
        float ha, la, hb, lb;
        spread_ends<M>(ala, ha, la);
        spread_ends<M>(alb, hb, lb);
        q2_pow1(ha, la, hb, lb, __uint_as_float(La * w23 + 0x3F800000u), __uint_as_float(Lb * w23 + 0x3F800000u), qa,
                qb);
    }

    // width_p2, also adding each field's fixed-point alpha (alpha_fx of the
    // same entry, from a second table `aoff` bytes after the first) to ax[m]
    __device__ __forceinline__ uint32_t width_p2_alpha(const float* v, uint32_t L, const uint32_t* cm, uint32_t aoff,
                                                       uint32_t (&ax)[M]) const
    {
        float al[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float t = mul_sat(__fsub_rn(v[m], lo[m]), s[m]);
            const uint32_t addr = __float_as_uint(fma_rz(t, Tf, 8388608.0f)) * 4u + cm[m];
            al[m] = lds_f32(addr);
            ax[m] += lds_u32(addr + aoff);
        }
        float f = importance<PM>(spread<M>(al), L, inv_vmax, mb, ma, wshift, n2, P);
        return __float2uint_rn(__fmul_rn(f, qscale));
    }

    // width from normalised values, also adding the fixed-point alphas
    // (s_ax: the u32 twin of the table s_tf)
    __device__ __forceinline__ uint32_t width_alpha(const float* t, uint32_t L, const float* s_tf,
                                                    const uint32_t* s_ax, uint32_t (&ax)[M]) const
    {
        float al[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const uint32_t e = m * T1 + floor_small(__fmul_rn(t[m], Tf));
            al[m] = s_tf[e];
            ax[m] += s_ax[e];
        }
        float f = importance<PM>(spread<M>(al), L, inv_vmax, mb, ma, wshift, n2, P);
        return __float2uint_rn(__fmul_rn(f, qscale));
    }
};

template <int M>
__device__ __forceinline__ void load_table(float* s_tf, const float* tf, uint32_t T)
{
    const uint32_t T1 = T + 1;
    for (uint32_t i = threadIdx.x; i < M * T1; i += blockDim.x) {
        uint32_t m = i / T1, e = i - m * T1;
        s_tf[i] = tf[m * T + (e < T ? e : T - 1)];
    }
}

// The fixed-point twin of load_table: s_ax[i] = alpha_fx(s_tf[i]).
template <int M>
__device__ __forceinline__ void load_table_fx(uint32_t* s_ax, const float* tf, uint32_t T)
{
    const uint32_t T1 = T + 1;
    for (uint32_t i = threadIdx.x; i < M * T1; i += blockDim.x) {
        uint32_t m = i / T1, e = i - m * T1;
        s_ax[i] = alpha_fx(tf[m * T + (e < T ? e : T - 1)]);
    }
}

// Loads 4 consecutive cells at idx (idx % 4 == 0; rows padded to 4 cells).
template <int M>
__device__ __forceinline__ void load4(const float* __restrict__ val, size_t pitch,
                                      const uint8_t* __restrict__ lev, uint64_t idx,
                                      float (&v)[4][M], uint32_t& L4)
{
#pragma unroll
    for (int m = 0; m < M; ++m) {
        float4 x = __ldg(reinterpret_cast<const float4*>(val + m * pitch + idx));
        v[0][m] = x.x; v[1][m] = x.y; v[2][m] = x.z; v[3][m] = x.w;
    }
    L4 = __ldg(reinterpret_cast<const uint32_t*>(lev + idx));
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Warp total of per-lane values below 2^35 (total below 2^40) with two redux adds.
__device__ __forceinline__ unsigned long long warp_total_small(unsigned long long x)
{
    unsigned lo = __reduce_add_sync(FULL, (unsigned)(x & 0xFFFFFFull));
    unsigned hi = __reduce_add_sync(FULL, (unsigned)(x >> 24));
    return ((unsigned long long)hi << 24) + lo;
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Pixel boundaries: C(k) = ceil(k F / W) is the first position of pixel k,
// D(k) = floor(k F / W); with F = a W + b, k F / W = k a + k b / W.
struct PixelMap {
    unsigned long long a, b, F;
    uint32_t W;
    __device__ __forceinline__ unsigned long long C(uint32_t k) const
    {
        unsigned long long kb = (unsigned long long)k * b;
        return (unsigned long long)k * a + (kb + W - 1) / W;
    }
    __device__ __forceinline__ unsigned long long D(uint32_t k) const
    {
        return (unsigned long long)k * a + ((unsigned long long)k * b) / W;
    }
    __device__ __forceinline__ uint32_t estimate(unsigned long long x) const
    {
        float e = __fmul_rn((float)x, __fdiv_rn((float)W, (float)F));
        uint32_t k = e > 0.0f ? (uint32_t)e : 0u;
        return k < W - 1 ? k : W - 1;
    }
    // pixel containing start position x: max{k < W : C(k) <= x}
    __device__ __forceinline__ uint32_t first_pixel(unsigned long long x) const
    {
        uint32_t k = estimate(x);
        while (k + 1 < W && C(k + 1) <= x) ++k;
        while (k > 0 && C(k) > x) --k;
        return k;
    }
    // last pixel touched by a span ending at I > start: max{k < W : D(k) <= I-1}
    __device__ __forceinline__ uint32_t last_pixel(unsigned long long I) const
    {
        unsigned long long y = I - 1;
        uint32_t k = estimate(y);
        while (k + 1 < W && D(k + 1) <= y) ++k;
        while (k > 0 && D(k) > y) --k;
        return k;
    }
};

}  // namespace
}  // namespace dvl
