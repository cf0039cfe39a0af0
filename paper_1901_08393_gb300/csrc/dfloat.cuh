// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, i.e. a 48-bit significand.  The error-free
// transformations of Knuth (two-sum), Dekker (fast two-sum) and the FMA two-product
// are written with explicit round-to-nearest intrinsics so that no compiler
// contraction or reassociation can break them.  On GB300 the FP32 pipe issues 64x
// the FP64 rate, so FP64-accurate arithmetic built this way runs far faster than
// native FP64 for the far-field quadrature and the dense V x.
#pragma once

#include <cuda_runtime.h>

namespace bem {

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// p + e = a * b exactly (FMA).
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Split an FP64 value into hi + lo (hi = nearest float, lo = nearest float to the rest).
__device__ __forceinline__ float2 df_from_double(double v)
{
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

__host__ __device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }

// (ah + al) + (bh + bl), renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    float h, l;
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
}

// a + b as df_add without the final renormalisation: hi is the rounded sum of the
// hi parts and lo collects the rest, so |lo| may exceed ulp(hi) / 2 by a few units
// of the lo parts' rounding.  For intermediate sums whose result goes through
// df_add (or df_to_double) before it is stored.
__device__ __forceinline__ float2 df_add_u(float2 a, float2 b)
{
    float s, e;
    two_sum(a.x, b.x, s, e);
    return make_float2(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

// (ah + al) * (bh + bl), renormalised.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    float p, e;
    two_prod(a.x, b.x, p, e);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float h, l;
    fast_two_sum(p, e, h, l);
    return make_float2(h, l);
}

}  // namespace bem
