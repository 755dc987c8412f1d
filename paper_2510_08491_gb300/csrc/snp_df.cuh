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

__device__ __forceinline__ f2 df_from(float a) { return {a, 0.0f}; }
__device__ __forceinline__ f2 df_neg(f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ f2 df_sub(f2 a, f2 b) { return df_add(a, df_neg(b)); }

// Exact product of two floats as a float-float value.
__device__ __forceinline__ f2 df_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ f2 df_mul_f(f2 a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_fast_two_sum(p, e);
}

// a / b: a first quotient, the float-float remainder a - q1 b, a correction.
__device__ __forceinline__ f2 df_div(f2 a, f2 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const f2 r = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_fast_two_sum(q1, q2);
}

// 1 / sqrt(a), a > 0: the MUFU estimate, then two Newton steps
// y <- y + y (1 - a y^2) / 2 in float-float (each step about doubles the bits).
__device__ __forceinline__ f2 df_rsqrt(f2 a)
{
    f2 y = df_from(rsqrtf(a.hi));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const f2 h = df_sub(df_from(1.0f), df_mul(a, df_mul(y, y)));
        y = df_add(y, df_mul_f(y, 0.5f * h.hi));
    }
    return y;
}

// exp(x) for a float x (|x| < 80): x = k ln2 + r with k = rint(x / ln2) and
// ln2 = L1 + L2 + L3 (L1 with 16 significant bits, so k L1 is exact; L2 + L3 the
// float-float remainder), |r| <= 0.35; exp(r) from its Maclaurin series to r^15
// (remainder < 1e-19) in float-float Horner form with 1/n! as float-float
// constants; then the exact scaling by 2^k.
__device__ __forceinline__ f2 df_exp(float x)
{
    constexpr float L1 = 0.693145751953125f, L2 = 1.4286068e-06f, L3 = 5.497923e-14f;
    const float k = rintf(x * 1.4426950216293335f);
    f2 r = df_two_sum(x, -k * L1);                  // x - k L1, exactly
    r = df_sub(r, df_mul(df_from(k), f2{L2, L3}));  // - k (L2 + L3)
    // 1/n!, n = 15 .. 0, as hi + lo
    const float ch[16] = {7.647163609812713e-13f, 1.147074536050896e-11f, 1.6059044372074283e-10f,
                          2.0876755879584152e-09f, 2.5052107943679403e-08f, 2.755731998149713e-07f,
                          2.7557318844628753e-06f, 2.4801587642286904e-05f, 0.00019841270113829523f,
                          0.0013888889225199819f, 0.008333333767950535f, 0.0416666679084301f,
                          0.1666666716337204f, 0.5f, 1.0f, 1.0f};
    const float cl[16] = {1.2200710471178288e-20f, 2.372207689231238e-19f, -5.352526511562726e-18f,
                          1.1082839147459852e-16f, 4.4176230446483665e-16f, -7.575112209051195e-15f,
                          3.793571224297229e-14f, -3.40699609366682e-13f, -2.725596874933456e-12f,
                          -3.3631094437103215e-11f, -4.34617203337595e-10f, -1.2417634698280722e-09f,
                          -4.967053879312289e-09f, 0.0f, 0.0f, 0.0f};
    f2 p{ch[0], cl[0]};
#pragma unroll
    for (int i = 1; i < 16; ++i) p = df_add(df_mul(p, r), f2{ch[i], cl[i]});
    const int ki = (int)k;
    return {ldexpf(p.hi, ki), ldexpf(p.lo, ki)};
}

}  // namespace snp
