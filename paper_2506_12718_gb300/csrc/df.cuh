// Double-float arithmetic: a real number as the unevaluated sum hi + lo of
// two FP32 values (about 48 significant bits), computed on the FP32 pipes.
//
// GB300 runs FP32 fused multiply-adds at 64 times its FP64 rate (128 against
// 2 per clock and SM), so an FFT that keeps FP64-level accuracy in pairs of
// FP32 values (about 15 FP32 instructions per FP64 operation) has several
// times the arithmetic throughput of the plain FP64 kernels.  The building
// blocks are the classical error-free transformations: the sum of two floats
// with its exact rounding error (Knuth's two-sum, 6 operations), the same
// when the larger operand is known (Dekker's fast two-sum, 3), and the exact
// error of a product from one fused multiply-add.  Every operation uses the
// explicitly rounded intrinsics (__fadd_rn, __fmaf_rn, ...), which the
// compiler neither contracts nor reorders.
//
//   a + b: two-sum of the high parts, the low parts added to its error, and a
//          fast two-sum to renormalise (11 operations); the error is bounded
//          by about 2^-46 (|a| + |b|), which is all an FFT's error analysis
//          needs (its butterflies are sums with bounded coefficients).
//   a * b: the high product, its exact error from a fused multiply-add, and
//          the two cross terms (4 operations, lo*lo dropped: below 2^-48).
//          The result is left unnormalised (|lo| below about 2^-22 |hi|);
//          every operation here accepts such operands, and the next sum
//          renormalises.
//
// Range: that of FP32 (normal numbers from about 1.2e-38 to 3.4e38), with
// the full 48 bits down to about 2^-102 (2e-31); below that the low part is
// subnormal and the precision falls gradually to FP32's.  The conversions
// from and to FP64 (df_from_double, df_to_double) keep that precision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pac {

struct __align__(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h) : hi(h), lo(0.f) {}  // NOLINT: implicit, as for float
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
};

// complex double-float, 16 bytes like double2: {re.hi, re.lo, im.hi, im.lo}
struct __align__(16) dfloat2 {
    dfloat x, y;
};

__device__ __forceinline__ dfloat df_fast_two_sum(float s, float e) {  // |s| >= |e| (or s = 0)
    const float h = __fadd_rn(s, e);
    return dfloat(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));  // s + e = a.hi + b.hi exactly
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // the exact error of p
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dfloat(p, e);
}

// FP64 -> double-float by integer operations on the bit pattern (no FP64
// instruction): hi = d with its significand truncated to 24 bits, lo = the
// remaining 29 bits (d - hi exactly), rounded to 24 bits.  Magnitudes below
// FP32's normal range give 0, above it infinity (a NaN stays a NaN).
__device__ __forceinline__ dfloat df_from_double(double d) {
    const uint32_t h = (uint32_t)__double2hiint(d), l = (uint32_t)__double2loint(d);
    const int ex = (int)((h >> 20) & 0x7ffu) - 1023;  // unbiased exponent
    const uint32_t sign = h & 0x80000000u;
    if (ex < -126) return dfloat(__uint_as_float(sign), 0.f);
    if (ex > 127) {  // infinity, or a quiet NaN for a NaN
        const bool nan = ex == 1024 && ((h & 0xfffffu) | l) != 0;
        return dfloat(__uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.f);
    }
    const float hi = __uint_as_float(sign | ((uint32_t)(ex + 127) << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
    // lo = (l mod 2^29) * 2^(ex - 52); the power of two is built in two
    // factors so that neither leaves FP32's range
    const float k = __uint2float_rn(l & 0x1fffffffu);
    const int e2 = ex - 52;  // in [-178, 75]
    const int e2a = e2 / 2, e2b = e2 - e2a;
    const float lo = __fmul_rn(__fmul_rn(k, __uint_as_float((uint32_t)(e2a + 127) << 23)),
                               __uint_as_float((uint32_t)(e2b + 127) << 23));
    return dfloat(hi, sign ? -lo : lo);
}

// FP32 -> FP64 exactly, by integer operations on the bit pattern (no FP64
// instruction) for normal numbers, infinities and NaNs; zero and subnormals
// (a low part below 2^-126, for values below about 2^-102) take the plain
// conversion.
__device__ __forceinline__ double df_widen(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t sign = b & 0x80000000u, ex = (b >> 23) & 0xffu, man = b & 0x7fffffu;
    if (ex == 0u) return (double)f;
    const uint32_t dex = ex == 0xffu ? 0x7ffu : ex + 896u;  // rebias 127 -> 1023
    return __hiloint2double((int)(sign | (dex << 20) | (man >> 3)), (int)(man << 29));
}

// double-float -> FP64: both parts widened exactly, one FP64 addition
__device__ __forceinline__ double df_to_double(dfloat a) { return df_widen(a.hi) + df_widen(a.lo); }

__device__ __forceinline__ dfloat2 df2_from_double2(double2 d) { return dfloat2{df_from_double(d.x), df_from_double(d.y)}; }
__device__ __forceinline__ double2 df2_to_double2(dfloat2 a) { return double2{df_to_double(a.x), df_to_double(a.y)}; }

}  // namespace pac
