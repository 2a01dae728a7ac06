// tm_df64.cuh -- double-float ("DF64") arithmetic: a real as the unevaluated sum hi + lo of two
// IEEE binary32 numbers with |lo| <= ulp(hi)/2, i.e. a 48-bit significand (relative rounding
// about 2^-48 = 3.6e-15).  Built from the classical error-free transformations:
//   TwoSum(a, b):  s = a + b and the exact error of that sum (Knuth, TAOCP vol. 2),
//   FastTwoSum(a, b), |a| >= |b|: the same with three operations (Dekker 1971),
//   TwoProd(a, b): p = a * b and its exact error fma(a, b, -p).
// On GB300 a binary32 FMA issues at many times the binary64 rate, so an operator evaluated in
// DF64 reaches double-precision-class accuracy at a multiple of the binary64 throughput.
//
// All binary32 steps use explicitly rounded operations so the compiler can neither contract nor
// reorder them (device: __fadd_rn & co.; host: plain float operations, compiled without
// contraction, for the CPU unit test).
#pragma once
#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace tmk {

// keep the binary32 / binary64 overloads visible next to the DF64 one below
using ::fma;

#ifdef __CUDA_ARCH__
__device__ __forceinline__ float df_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float df_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float df_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float df_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float df_add(float a, float b) { volatile float r = a + b; return r; }
inline float df_sub(float a, float b) { volatile float r = a - b; return r; }
inline float df_mul(float a, float b) { volatile float r = a * b; return r; }
inline float df_fma(float a, float b, float c) { return fmaf(a, b, c); }
#endif

struct df64 {
    float hi, lo;
    __host__ __device__ df64() : hi(0.f), lo(0.f) {}
    __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
    // from a binary64 value: hi = nearest float, lo = nearest float to the exact remainder
    __host__ __device__ explicit df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit df64(int v) : df64((double)v) {}
    __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

__host__ __device__ __forceinline__ df64 two_sum(float a, float b)
{
    const float s = df_add(a, b);
    const float bb = df_sub(s, a);
    const float e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
    return df64(s, e);
}
__host__ __device__ __forceinline__ df64 fast_two_sum(float a, float b)
{
    const float s = df_add(a, b);
    return df64(s, df_sub(b, df_sub(s, a)));
}
__host__ __device__ __forceinline__ df64 two_prod(float a, float b)
{
    const float p = df_mul(a, b);
    return df64(p, df_fma(a, b, -p));
}

// sum: exact sum of the high parts, plus the low parts, renormalised once.  The error is a few
// 2^-48 relative to |a| + |b| (not to |a + b| under cancellation), which is what a sum of
// similar-sized stencil terms needs, at 11 operations instead of the 20 of the fully
// renormalised form.
__host__ __device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    df64 s = two_sum(a.hi, b.hi);
    s.lo = df_add(s.lo, df_add(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
// product: exact product of the high parts plus the two cross terms (lo*lo is below 2^-48)
__host__ __device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    df64 p = two_prod(a.hi, b.hi);
    p.lo = df_fma(a.hi, b.lo, p.lo);
    p.lo = df_fma(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
__host__ __device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__host__ __device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }
// a * b + c with the product kept unrounded until the sum (error a few 2^-48 relative to
// |a b| + |c|; 15 operations)
__host__ __device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c)
{
    df64 p = two_prod(a.hi, b.hi);
    p.lo = df_fma(a.hi, b.lo, p.lo);
    p.lo = df_fma(a.lo, b.hi, p.lo);
    df64 s = two_sum(p.hi, c.hi);
    s.lo = df_add(s.lo, df_add(p.lo, c.lo));
    return fast_two_sum(s.hi, s.lo);
}

}  // namespace tmk
