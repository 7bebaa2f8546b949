// Double-float arithmetic on the float32 pipe (internal).
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2: about 44
// significant bits.  Built from the error-free transformations of the literature: the
// two-sum of Knuth (TAOCP vol. 2, Sec. 4.2.2), Dekker's fast two-sum (Numer. Math. 18,
// 1971) and the two-product through a fused multiply-add.  Every step is written with the
// round-to-nearest intrinsics, which the compiler neither contracts into fused operations
// nor reassociates, so each transformation is exact as written.
//
// Used where float32 cannot hold a difference of two large terms to the required absolute
// accuracy and float64 is too slow on this part (about 2 float64 FMA per clock per SM
// against 128 float32 FMA).
#pragma once

#include <cuda_runtime.h>

namespace rift {

struct df {
    float hi, lo;
};

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// a + b = s + e exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ df df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df a, df b)
{
    const df s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }

// product: the rounding error of hi*hi by a fused multiply-add, the cross terms added to
// it (lo*lo is below the format's precision)
__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mac(df acc, df a, df b) { return df_add(acc, df_mul(a, b)); }

// acc += a b for a long sum: the product's rounding error and cross terms, and the
// rounding error of adding its high part, collect in acc.lo without renormalising (the
// running high part depends on the previous one through a single addition, so independent
// sums interleave well); df_norm once at the end.
__device__ __forceinline__ void df_acc(df &acc, df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df s = df_two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}

__device__ __forceinline__ df df_norm(df a) { return df_two_sum(a.hi, a.lo); }

__device__ __forceinline__ df df_of(double v)
{
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_shfl_xor(df a, int o)
{
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// complex double-float
struct dfc {
    df re, im;
};

__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b)
{
    return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}

}  // namespace rift
