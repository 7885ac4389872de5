// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significant bits.  The error-free transformations are
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971) and TwoProduct through a
// fused multiply-add; the sums and products below are the standard double-word algorithms
// built from them (Dekker 1971; Joldes, Muller & Popescu, "Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic", ACM TOMS 2017).  They run on the
// FP32 pipes, which on GB300 issue ~64x the FP64 rate.
#pragma once

#include <cuda_runtime.h>

namespace labfm {

// 8-byte aligned, so that a value in shared or global memory moves as one 64-bit access (two
// 32-bit accesses of a warp split across the banks conflict wherever rows are an even number
// of words apart).  Every array of df starts on an 8-byte boundary.
struct __align__(8) df {
    float hi, lo;
};
static_assert(sizeof(df) == 8 && alignof(df) == 8, "double-float layout");

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// exact split of a double into hi + lo (the rounding error of lo is below 2^-48 |x|)
__device__ __forceinline__ df df_from_double(double x)
{
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df{h, l};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, provided |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e = a * b exactly (barring underflow)
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e, t, f;
    two_sum(a.hi, b.hi, s, e);
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return df{s, e};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_mul(df a, df b)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    fast_two_sum(p, e, p, e);
    return df{p, e};
}

// acc + a * b
__device__ __forceinline__ df df_fma(df a, df b, df acc)
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(acc.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(acc.lo, e));
    fast_two_sum(s, t, s, t);
    return df{s, t};
}

// acc - a * b
__device__ __forceinline__ df df_fms(df a, df b, df acc) { return df_fma(df_neg(a), b, acc); }

// 1 / b: float seed, then one Newton step y + y (1 - b y) in double-float
__device__ __forceinline__ df df_recip(df b)
{
    float y = __frcp_rn(b.hi);
    df one_minus = df_fma(df_neg(b), df{y, 0.0f}, df{1.0f, 0.0f});
    df corr = df_mul(df{y, 0.0f}, one_minus);
    float s, e;
    fast_two_sum(y, corr.hi, s, e);
    e = __fadd_rn(e, corr.lo);
    fast_two_sum(s, e, s, e);
    return df{s, e};
}

__device__ __forceinline__ float df_abs_hi(df a) { return fabsf(a.hi); }
__device__ __forceinline__ bool df_isfinite(df a) { return isfinite(a.hi) && isfinite(a.lo); }

}  // namespace labfm
