// Bit-level helpers for IEEE doubles on GB300 (sm_103a).
//
// On this part every FP64 instruction -- arithmetic, compares, min/max and
// conversions alike -- issues to a narrow FP64 unit (2 thread-operations per
// clock per SM), so these helpers do compares, conversions and the reciprocal
// seed with integer and single-precision instructions instead.
#pragma once

#include <cuda_runtime.h>

namespace l2x {

// ---------------------------------------------------------------- bit-level helpers
// On GB300 every FP64 instruction (compare, min/max and conversion included) runs
// on the narrow FP64 unit; these helpers do the same jobs with integer
// instructions on the bit patterns of IEEE doubles (finite inputs only).

// Signed-integer key with the same order as the doubles it encodes.
__device__ __forceinline__ long long order_key(double x) {
    long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double from_order_key(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
// x >= y (with -0.0 < +0.0, a consistent tie rule for both sides of every plane)
__device__ __forceinline__ bool ge_d(double x, double y) { return order_key(x) >= order_key(y); }
__device__ __forceinline__ bool le_d(double x, double y) { return order_key(x) <= order_key(y); }
// sign bit clear: x >= +0.0
__device__ __forceinline__ bool nonneg_d(double x) { return __double2hiint(x) >= 0; }

// double -> float, rounding half away from zero in magnitude, flushing magnitudes
// below 2^-126 to zero (the moment arithmetic never needs subnormals).
__device__ __forceinline__ float d2f_int(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x) + 0x10000000ull;
    unsigned int hi = (unsigned int)(b >> 32);
    int e = (int)((hi >> 20) & 0x7ff) - 896;
    unsigned int sign = hi & 0x80000000u;
    if (e <= 0) return __uint_as_float(sign);
    unsigned int m = (unsigned int)(b >> 29) & 0x7fffffu;
    return __uint_as_float(sign | ((unsigned int)e << 23) | m);
}
// float -> double, exact (normal floats; zero maps to zero).
__device__ __forceinline__ double f2d_int(float f) {
    unsigned int u = __float_as_uint(f);
    unsigned int e = (u >> 23) & 0xff;
    if (e == 0) return __longlong_as_double((long long)(u & 0x80000000u) << 32);
    unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                           ((unsigned long long)(e + 896) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

template <typename R>
__device__ __forceinline__ R to_r(double x);
template <>
__device__ __forceinline__ double to_r<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_r<float>(double x) { return d2f_int(x); }

// a / b by Newton's iteration for the reciprocal: an FP32 seed (24 bits), two
// refinements r <- r + r (1 - b r) (48, then more than 53 bits: the rounding of
// r is what remains), and the product q = a r, within two ulps of the correctly
// rounded quotient (the iteration is the one P. Markstein's division builds on,
// "Computation of elementary functions on the IBM RISC System/6000 processor",
// IBM J. Res. Dev. 34(1), 1990; his final correction of q, two more FP64
// operations, is left out: the clipping needs the crossing parameter to FP64
// accuracy, not correctly rounded).  Used for the edge parameters of plane
// crossings, where |b| > 0 and a / b lies in [0, 1], and the CG's scalars;
// operands far from 1 in magnitude take the hardware division.
__device__ __forceinline__ double div_nr(double a, double b) {
    const int eb = (__double2hiint(b) >> 20) & 0x7ff;
    if (eb < 1023 - 120 || eb > 1023 + 120) return a / b;
    double r = f2d_int(__frcp_rn(d2f_int(b)));
    double e = fma(-b, r, 1.0);
    r = fma(r, e, r);
    e = fma(-b, r, 1.0);
    r = fma(r, e, r);
    return a * r;
}

// a / b to about 2^-45 relative with two FP64 instructions, for the crossing
// parameters of the mixed precision form: the FP32 quotient t0 = a r0 (r0 the
// FP32 reciprocal of b) and one correction t0 + (a - t0 b) r0, the residual of
// t0 times the approximate reciprocal (the Newton step for the quotient, as in
// the division of Markstein 1990 cited above).  The step squares the relative
// error of t0 (a few 2^-24) times that of r0.  |b| > 0; operands far from 1 in
// magnitude take the hardware division.
__device__ __forceinline__ double div_fast(double a, double b) {
    const int eb = (__double2hiint(b) >> 20) & 0x7ff;
    if (eb < 1023 - 120 || eb > 1023 + 120) return a / b;
    const float rf = __frcp_rn(d2f_int(b));
    const double r0 = f2d_int(rf);
    const double t0 = f2d_int(__fmul_rn(d2f_int(a), rf));
    return fma(fma(-t0, b, a), r0, t0);
}

// x * 2^e for x = 0 or x * 2^e and x both normal: one integer add on the
// exponent field of the high word (zero stays zero)
__device__ __forceinline__ double ldexp_normal_int(double x, int e) {
    const int hi = __double2hiint(x);
    return __hiloint2double(hi + ((hi & 0x7ff00000) ? (e << 20) : 0), __double2loint(x));
}

// non-negative int -> double, exact, by integer instructions
__device__ __forceinline__ double i2d_int(int v) {
    if (v <= 0) return 0.0;
    const int e = 31 - __clz(v);
    const unsigned long long m = ((unsigned long long)(unsigned int)v << (52 - e)) & 0x000fffffffffffffull;
    return __longlong_as_double((long long)(((unsigned long long)(1023 + e) << 52) | m));
}


// Double-float value (hi + lo) and its sum with a second one (Knuth's two-sum,
// renormalised); single-precision instructions only.
struct __align__(8) DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
    const float h = __fadd_rn(s, lo);
    return DF{h, __fsub_rn(lo, __fsub_rn(h, s))};
}

// Product of two double-float values, left unnormalised (|lo| stays within a few
// ulps of |hi|): hi*hi exactly by the FMA two-product, plus the cross terms; the
// dropped lo*lo term is below 2^-46 of the product.
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return DF{p, e};
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

__device__ __forceinline__ DF df_from_double(double x) {
    const float hi = d2f_int(x);
    return DF{hi, d2f_int(x - f2d_int(hi))};
}

__device__ __forceinline__ double df_to_double(DF a) { return f2d_int(a.hi) + f2d_int(a.lo); }

// x * 2^e by integer arithmetic on the exponent field (finite x; results below
// the normal range become zero of the same sign).
__device__ __forceinline__ float ldexp_f_int(float x, int e) {
    const unsigned int u = __float_as_uint(x);
    const int ex = (int)((u >> 23) & 0xff);
    if (ex == 0) return __uint_as_float(u & 0x80000000u);
    const int en = ex + e;
    if (en <= 0) return __uint_as_float(u & 0x80000000u);
    return __uint_as_float((u & 0x807fffffu) | ((unsigned int)en << 23));
}
__device__ __forceinline__ double ldexp_d_int(double x, int e) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7ff);
    if (ex == 0) return __longlong_as_double((long long)(u & 0x8000000000000000ull));
    const int en = ex + e;
    if (en <= 0) return __longlong_as_double((long long)(u & 0x8000000000000000ull));
    return __longlong_as_double((long long)((u & 0x800fffffffffffffull) | ((unsigned long long)en << 52)));
}
// The low part of the double-float split of x whose high part is d2f_int(x):
// x - d2f_int(x) as a float, by integer instructions only.  d2f_int keeps the top
// 24 mantissa bits, rounding on bit 28, so the remainder is the low 29 bits read
// as a signed number of ulps of x; its top 23 bits are kept (the split then
// holds 47 or more significant bits of x).  Zero where d2f_int flushes to zero.
__device__ __forceinline__ float d2f_lo_int(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    int r = ((int)((unsigned int)(b & 0x1fffffffull) << 3)) >> 3;  // x - hi in ulps of x, in [-2^28, 2^28)
    if (r == 0 || e <= 896) return 0.0f;
    unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    if (r < 0) {
        r = -r;
        sign ^= 0x80000000u;
    }
    const unsigned int a = (unsigned int)r;
    const int sh = max(0, 9 - __clz(a));  // a >> sh < 2^23
    const float f = __fsub_rn(__uint_as_float(0x4b000000u | (a >> sh)), 8388608.0f);  // exactly a >> sh
    return ldexp_f_int(__uint_as_float(__float_as_uint(f) | sign), sh + e - 1075);
}
__device__ __forceinline__ DF df_split_int(double x) { return DF{d2f_int(x), d2f_lo_int(x)}; }

// binary exponent of a positive finite double (floor(log2 x))
__device__ __forceinline__ int ilogb_int(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}
__device__ __forceinline__ DF df_scale(DF a, int e) { return DF{ldexp_f_int(a.hi, e), ldexp_f_int(a.lo, e)}; }

__device__ __forceinline__ DF df_shfl_xor(DF a, int o) {
    return DF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

}  // namespace l2x
