// snp_df.cuh -- float-float arithmetic on the FP32 pipe: a value is hi + lo with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  Built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971)
// and the FMA form of TwoProduct (the rounding error of a*b is fma(a, b, -a*b)).
// Every operation is an explicitly rounded intrinsic, so the compiler cannot
// contract or reorder the steps the transformations rely on.
//
// Error model used by the callers: the sum of two float-float values is exact
// up to ~2^-47 (|a| + |b|) (the "sloppy" sum: its error is relative to the
// inputs, not to a result that cancels to near zero, which is what a caller
// evaluating a polynomial near one of its roots needs), the product up to
// ~2^-47 |a b|.
#pragma once

#include <cuda_runtime.h>

namespace snp {

struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ f2 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ f2 df_add(f2 a, f2 b)
{
    const f2 s = df_two_sum(a.hi, b.hi);
    // TwoSum, not FastTwoSum, for the renormalisation: after cancellation the
    // correction can exceed the leading part
    return df_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ f2 df_mul(f2 a, f2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

}  // namespace snp
