// Per-field log10 value scale, applied when the values are gathered into
// curve order so that every kernel after it sees the scaled field.
//
// Fields that span many decades (densities, pressures of astrophysical AMR
// data) are normalised on a log axis; the paper normalises each field by its
// own domain before the transfer function (Sec. 3.3), and this transform comes
// before that normalisation.  A log-scaled value v becomes log10(v); v <= 0
// first takes the field's smallest positive value.
//
// log10 of x > 0, as a fixed sequence of correctly rounded float32 operations
// (explicit _rn intrinsics, no contraction), so that every IEEE float32
// implementation of the same sequence returns the same bits:
//   x = m 2^e, m in [s/2, s) with s = float32(sqrt 2); a subnormal x is first
//     multiplied by 2^24 (exact);
//   z = (m - 1) / (m + 1), kept as z + dz with dz the quotient's residual
//     (fma) over m + 1, whose rounding error dlo is itself exact;
//   log10 m = 2 log10(e) atanh(z) = (z + dz) (c0 + c1 z^2 + ... + c4 z^8),
//     c_k = 2 log10(e) / (2k + 1) from the Taylor series of atanh, cut where
//     the next term is below 0.05 ulp (|z| <= 0.1716);
//   log10 x = e h + (e l + log10 m) with h + l = log10(2), h of 16 bits so
//     that e h is exact.
// Error: within 1.5 ulp of the exact log10 for every positive float.
#pragma once

#include <cstdint>

namespace dvl {

__device__ __forceinline__ float log10_scale(float x)
{
    const float c0 = 0x1.bcb7b2p-1f, c1 = 0x1.287a76p-2f, c2 = 0x1.63c628p-3f, c3 = 0x1.fc3fa6p-4f,
                c4 = 0x1.8b4df2p-4f;
    const float l2_hi = 0x1.344p-2f, l2_lo = 0x1.3509f8p-18f;
    const float s2 = 0x1.6a09e6p+0f;
    int e = 0;
    if (x < 0x1p-126f) { x = __fmul_rn(x, 0x1p24f); e = -24; }
    uint32_t b = __float_as_uint(x);
    e += (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m >= s2) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float num = __fsub_rn(m, 1.0f);
    const float den = __fadd_rn(m, 1.0f);
    const float dlo = __fsub_rn(m, __fsub_rn(den, 1.0f));
    const float z = __fdiv_rn(num, den);
    float r = __fmaf_rn(-z, den, num);
    r = __fmaf_rn(-z, dlo, r);
    const float dz = __fdiv_rn(r, den);
    const float w = __fmul_rn(z, z);
    float p = c4;
    p = __fmaf_rn(p, w, c3);
    p = __fmaf_rn(p, w, c2);
    p = __fmaf_rn(p, w, c1);
    p = __fmaf_rn(p, w, c0);
    const float lm = __fmaf_rn(z, p, __fmul_rn(dz, c0));
    const float ef = (float)e;
    return __fmaf_rn(ef, l2_hi, __fmaf_rn(ef, l2_lo, lm));
}

}  // namespace dvl
