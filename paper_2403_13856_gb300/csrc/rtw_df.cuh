// rtw_df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of two
// single-precision numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.  On GB300 a
// single-precision operation issues at 64 times the double-precision rate, so the ten to thirty
// single-precision operations of one double-float operation cost less than one FP64 operation.
//
// The operations follow the published error-free transformations: Knuth's TwoSum, Dekker's
// Fast2Sum (|a| >= |b|), the FMA form of TwoProduct, and the double-double algorithms of Hida,
// Li and Bailey (accurate addition, multiplication, division by two correction quotients, square
// root by one Newton step).  Every step uses the _rn intrinsics so that the compiler neither fuses
// nor reorders them.  The exponent range is that of single precision (about 1e-38 .. 3e38).
#pragma once

#include <cuda_runtime.h>

namespace rtw {

// the double-float overloads below must not hide the standard ones inside this namespace
using ::copysign;
using ::fabs;
using ::rsqrt;
using ::sqrt;

struct df {
    float hi, lo;
    __device__ __forceinline__ df() : hi(0.0f), lo(0.0f) {}
    __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit df(int v) : hi((float)v), lo(0.0f) {}
    __device__ __forceinline__ explicit df(float v) : hi(v), lo(0.0f) {}
    __device__ __forceinline__ explicit df(double v)
    {
        hi = __double2float_rn(v);
        lo = __double2float_rn(v - (double)hi);
    }
    __device__ __forceinline__ operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df operator+(const df& a, const df& b)
{
    float s, e, t, f;
    df_two_sum(a.hi, b.hi, s, e);
    df_two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    df_fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    df_fast_two_sum(s, e, s, e);
    return df(s, e);
}

__device__ __forceinline__ df operator-(const df& a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(const df& a, const df& b) { return a + (-b); }

__device__ __forceinline__ df operator*(const df& a, const df& b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s;
    df_fast_two_sum(p, e, s, e);
    return df(s, e);
}

// a * b with b a single-precision number
__device__ __forceinline__ df df_mul_f(const df& a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    float s;
    df_fast_two_sum(p, e, s, e);
    return df(s, e);
}

__device__ __forceinline__ df operator/(const df& a, const df& b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    df r = a - df_mul_f(b, q1);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    r = r - df_mul_f(b, q2);
    const float q3 = __fdiv_rn(r.hi, b.hi);
    float s, e;
    df_fast_two_sum(q1, q2, s, e);
    return df(s, e) + df(q3);
}

__device__ __forceinline__ df& operator+=(df& a, const df& b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, const df& b) { return a = a - b; }
__device__ __forceinline__ df& operator*=(df& a, const df& b) { return a = a * b; }

__device__ __forceinline__ bool operator<(const df& a, const df& b)
{
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(const df& a, const df& b) { return b < a; }
__device__ __forceinline__ bool operator<=(const df& a, const df& b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(const df& a, const df& b) { return !(a < b); }
__device__ __forceinline__ bool operator==(const df& a, const df& b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(const df& a, const df& b) { return !(a == b); }

__device__ __forceinline__ df fabs(const df& a) { return (a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f)) ? -a : a; }

__device__ __forceinline__ df copysign(const df& a, const df& b)
{
    const bool neg = b.hi < 0.0f || (b.hi == 0.0f && (b.lo < 0.0f || signbit(b.hi)));
    const df m = fabs(a);
    return neg ? -m : m;
}

// one Newton step x + (a - x^2) / (2 x) from the single-precision root
__device__ __forceinline__ df sqrt(const df& a)
{
    if (!(a.hi > 0.0f)) return df(0.0f, 0.0f);
    const float x = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(x, x);
    const float pe = __fmaf_rn(x, x, -p);
    // a - x^2 in double-float, then the correction in single precision
    const df r = a - df(p, pe);
    const float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, x));
    float s, e;
    df_fast_two_sum(x, c, s, e);
    return df(s, e);
}

// 1 / sqrt(a): one Newton step y + y (1 - a y^2) / 2 from the single-precision estimate
__device__ __forceinline__ df rsqrt(const df& a)
{
    const float y = rsqrtf(a.hi);
    const df t = df_mul_f(df_mul_f(a, y), y);  // a y^2, close to 1
    const df h = df(1.0f) - t;
    const float c = __fmul_rn(__fmul_rn(0.5f, y), h.hi);
    float s, e;
    df_fast_two_sum(y, c, s, e);
    return df(s, e);
}

}  // namespace rtw
