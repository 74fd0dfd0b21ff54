// Double-single arithmetic for the FP64 plans: a value carried as an unevaluated
// sum hi + lo of two FP32 numbers (|lo| <= ulp(hi) / 2, 48 significant bits),
// so that FP64-accurate work runs on the FP32 units, which GB300 has at 64 times
// its FP64 rate.  Error-free transformations (Knuth's TwoSum, the FMA-based
// TwoProduct) and the compensated dot product of Ogita, Rump and Oishi (Dot2):
// a sum of products accumulated this way carries an error of about
// (n u)^2 sum |x_i y_i| (u = 2^-24) before its final rounding.  The operations
// use the _rn intrinsics so that no product is contracted into a neighbouring
// addition, which would break the transformations.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

// (global namespace: the complex overloads must join the generic cmake / cmul
// of common.cuh in the same overload set)

struct df32 {
    float hi, lo;
    __host__ __device__ constexpr df32() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    // constants (folded at compile time); not for values computed at run time
    __host__ __device__ constexpr df32(double d)
        : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr df32(int i) : df32((double)i) {}
};

// s + e = a + b exactly.
__device__ __forceinline__ df32 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0).
__device__ __forceinline__ df32 quick_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * s + c in double-single (one Horner step).
__device__ __forceinline__ df32 df_mul_add(df32 a, df32 s, df32 c) {
    const float p = __fmul_rn(a.hi, s.hi);
    float e = fmaf(a.hi, s.hi, -p);
    e = fmaf(a.hi, s.lo, e);
    e = fmaf(a.lo, s.hi, e);
    df32 t = two_sum(p, c.hi);
    t.lo = __fadd_rn(t.lo, __fadd_rn(e, c.lo));
    return quick_two_sum(t.hi, t.lo);
}

// Arithmetic on double-single values ("sloppy" addition: the low parts are
// added without their own error term, which keeps normwise accuracy of about
// u^2 for the FFT's butterflies), complex numbers of two of them, and the
// helpers the FFT engine uses (cmake, cmul, twiddle loads).
__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
    df32 s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }
__device__ __forceinline__ df32 operator*(df32 a, df32 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}

struct dfc {
    df32 x, y;
};
__device__ __forceinline__ dfc cmake(df32 a, df32 b) { return dfc{a, b}; }
__device__ __forceinline__ dfc operator+(dfc a, dfc b) { return dfc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dfc operator-(dfc a, dfc b) { return dfc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dfc cmul(dfc a, dfc b) {
    return dfc{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// A complex FP64 value (user data) as double-single.
__device__ __forceinline__ dfc to_dfc(double2 v);
// Read-only loads of table entries.
__device__ __forceinline__ dfc ldt(const dfc *p) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return dfc{df32(v.x, v.y), df32(v.z, v.w)};
}
__device__ __forceinline__ float2 ldt(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ldt(const double2 *p) { return __ldg(p); }

// One term of a compensated dot product: (r, c) += x * y with x, y double-single;
// r is the running FP32 sum, c collects the rounding errors and the low parts.
__device__ __forceinline__ void dot2_step(float &r, float &c, df32 x, df32 y) {
    const float p = __fmul_rn(x.hi, y.hi);
    const float e = fmaf(x.hi, y.hi, -p);
    const df32 t = two_sum(r, p);
    r = t.hi;
    c = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, __fadd_rn(c, __fadd_rn(t.lo, e))));
}

// A double as hi + lo: hi holds the top 24 bits of the significand (truncated),
// lo the remaining 29 rounded to 24, by integer operations on the bit pattern
// (no FP64 arithmetic).  Magnitudes outside [2^-100, 2^100) take the plain
// conversion.
__device__ __forceinline__ df32 split_double(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 1023 - 100 || e >= 1023 + 100) return {__double2float_rn(v), 0.f};
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned long long m = b & 0xfffffffffffffULL;
    const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) |
                                     (unsigned)(m >> 29));
    // lo = (m mod 2^29) 2^(e - 1075), scaled in two exact steps
    const float r = __uint2float_rn((unsigned)(m & 0x1fffffffULL));
    const float s1 = __uint_as_float((unsigned)(e - 1075 + 64 + 127) << 23);   // 2^(e - 1011)
    const float lo = __fmul_rn(__fmul_rn(r, 0x1p-64f), s1);     // stays inside FP32's range
    return {hi, sign ? -lo : lo};
}

__device__ __forceinline__ dfc to_dfc(double2 v) {
    return dfc{split_double(v.x), split_double(v.y)};
}

// Exponent scaling of the double-single passes.  FP32 covers 2^-126 .. 2^128
// and split_double keeps a low part only inside [2^-100, 2^100), while a
// caller's FP64 coefficients may sit anywhere in FP64's range.  So every line
// (member x field) is carried as c 2^-s, with s = emax - 1023 and emax the
// largest biased FP64 exponent among the coefficients the theta pass reads:
// the largest coefficient then lies in [1, 2) whatever the caller's units, and
// the interpolated values are multiplied back by 2^s.  Both scalings are exact
// (powers of two), so a field and the same field times 2^k give values that
// differ by exactly 2^k.  A line of zeros or subnormals (emax = 0), or one
// holding a non-finite value (emax = 0x7ff), keeps s = 0.
__device__ __forceinline__ int df_line_shift(int emax) {
    return (emax <= 0 || emax >= 0x7ff) ? 0 : emax - 1023;
}

// v 2^-s: the exponent field lowered by integer arithmetic when the result is
// a normal number (every value within 2^1022 of the line's largest), else a
// multiplication by the power of two (zeros, subnormals, non-finite values and
// results below the normal range).  s in [-1022, 1023].
__device__ __forceinline__ double df_scale_down(double v, int s) {
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e >= 1 && e < 0x7ff && e - s >= 1 && e - s < 0x7ff)
        return __longlong_as_double(b - ((long long)s << 52));
    return scalbn(v, -s);
}

// 2^s as a double, s in [-1022, 1023].
__device__ __forceinline__ double df_pow2(int s) {
    return __longlong_as_double((long long)(s + 1023) << 52);
}

// A complex FP64 coefficient of a line with shift s, as double-single.
__device__ __forceinline__ dfc to_dfc_scaled(double2 v, int s) {
    return dfc{split_double(df_scale_down(v.x, s)), split_double(df_scale_down(v.y, s))};
}

template <> struct CxT<df32> { typedef dfc type; };
