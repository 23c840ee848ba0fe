// Per-TF constants of an update, shared by the single-TF and the batched
// kernels: TF domains, the Eq. 5 entry range, the Eq. 6 max-variation
// approximation and the fixed-point exponent Q.  Included by .cu files only.
#pragma once

#include "cell_math.cuh"

namespace dvl {
namespace {

// ---------------------------------------------------------------------------
// Constants (Sec. 3.4 and the fixed-point exponent)
// ---------------------------------------------------------------------------

__device__ int bitlen64(uint64_t x) { return x ? 64 - __clzll((long long)x) : 0; }

// f_upper, Q, 2^Q from vmax (after vmax is known).
__device__ void finish_consts(UpdateConsts* C, const UpdateArgs& a, uint32_t max_level)
{
    const float vmax = C->vmax;
    const float inv = vmax > 0.0f ? __frcp_rn(vmax) : 0.0f;
    C->inv_vmax = inv;
    const bool after = C->min_imp_mode == DVL_MINIMP_AFTER_POWER;
    float fu = importance<POW_GEN>(vmax > 0.0f ? 1.0f : 0.0f, max_level, inv, after ? 0.0f : C->min_imp,
                                   after ? C->min_imp : 0.0f, C->width_shift, C->pow_n2, C->P);
    C->f_upper = fu;
    int Q = 0;
    if (!isfinite(fu)) {
        atomicOr(a.err, ERR_RANGE);
    } else {
        int e = 0;
        frexpf(fu, &e);                       // fu <= 2^e
        if (C->pow_n2 < 0) e += 1;            // powf is not monotone to the ulp
        int cap = 62 - bitlen64(a.n);         // total below 2^62
        if (cap > 31) cap = 31;               // every width below 2^32
        Q = cap - e;
        if (Q > 120) Q = 120;
        if (Q < -120) { atomicOr(a.err, ERR_RANGE); Q = 0; }
    }
    C->Q = Q;
    C->qscale = exp2i(Q);
    C->F = 0;
    C->linear = 0;
}

// Per-TF constants (one block of 256 threads): TF domains, Eq. 5 entry range,
// Eq. 6 max-variation approximation and the fixed-point exponent.
__device__ void prepare_consts_block(const UpdateArgs& a)
{
    __shared__ int s_i[DVL_MAX_FIELDS], s_j[DVL_MAX_FIELDS];
    __shared__ float s_spread[256];
    UpdateConsts* C = a.consts;
    const uint32_t M = a.M, T = a.T;
    const int tid = threadIdx.x;
    if (tid == 0) {
        C->P = a.prm.P;
        C->min_imp = a.prm.min_importance;
        C->min_imp_mode = (int)a.prm.min_imp_mode;
        C->width_shift = a.prm.width_mode == DVL_WIDTH_VOLUME ? 3 : 1;
        float n2 = 2.0f * a.prm.P;
        C->pow_n2 = (n2 >= 0.0f && n2 <= 16.0f && floorf(n2) == n2) ? (int)n2 : -1;
    }
    if (tid < (int)M) {
        float dmin = ordered_to_float(a.meta->dmin[tid]);
        float dmax = ordered_to_float(a.meta->dmax[tid]);
        if (a.n == 0) { dmin = 0.0f; dmax = 0.0f; }
        float lo = a.dom[tid], hi = a.dom[M + tid];
        if (isnan(lo) && isnan(hi)) { lo = dmin; hi = dmax; }
        float span = __fsub_rn(hi, lo);
        float s = (span > 0.0f && isfinite(span)) ? __frcp_rn(span) : 0.0f;
        // s = 0 maps every value to t = 0; lo = 0 keeps (v - lo) * s finite
        // (a range wider than the float range would otherwise give inf * 0)
        lo = s == 0.0f ? 0.0f : lo;
        C->lo[tid] = lo;
        C->s[tid] = s;
        // Eq. 5: TF entries of the data minimum and maximum of this field
        s_i[tid] = (int)tf_entry(norm_t(dmin, lo, s), (float)T, T - 1);
        s_j[tid] = (int)tf_entry(norm_t(dmax, lo, s), (float)T, T - 1);
    }
    __syncthreads();
    int gi = (int)T - 1, gj = 0;
    for (uint32_t m = 0; m < M; ++m) { gi = min(gi, s_i[m]); gj = max(gj, s_j[m]); }
    if (gi > gj) { gi = 0; gj = 0; }
    // Eq. 6: largest spread max_m A(m,a) - min_m A(m,a) over a in [gi, gj]
    float best = 0.0f;
    for (int e = gi + tid; e <= gj; e += blockDim.x) {
        float hi = a.tf[e], lw = a.tf[e];
        for (uint32_t m = 1; m < M; ++m) {
            float x = a.tf[m * T + e];
            hi = fmaxf(hi, x);
            lw = fminf(lw, x);
        }
        best = fmaxf(best, __fsub_rn(hi, lw));
    }
    s_spread[tid] = best;
    __syncthreads();
    if (tid == 0) {
        C->i = gi;
        C->j = gj;
        if (a.prm.vmax_mode == DVL_VMAX_APPROX) {
            float v = 0.0f;
            for (int k = 0; k < (int)blockDim.x; ++k) v = fmaxf(v, s_spread[k]);
            C->vmax = v;
            finish_consts(C, a, a.meta->max_level);
        } else {
            C->vmax = 0.0f;   // filled by k_vmax_exact, then k_consts
        }
    }
}

}  // namespace
}  // namespace dvl
