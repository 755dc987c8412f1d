// snp_mma.cuh -- warp-level tensor-core helpers (mma.sync m16n8k16 with bf16
// inputs and FP32 accumulation, ldmatrix, movmatrix) for the per-primitive
// colour-MLP contractions of a warp batch of 32 pixel rays.
//
// FP32 operands are split into bf16 pairs x = hi + lo (hi = bf16(x), lo =
// bf16(x - hi)); a product is accumulated as hi*hi + hi*lo + lo*hi, which keeps
// about 16 significant bits of each operand (relative error near 2^-16 per
// product rather than the 2^-8 of plain bf16).  Operands that are exactly bf16
// (weights stored in bf16) have lo = 0 and skip their correction product.
//
// Fragment layouts (PTX ISA, m16n8k16 .bf16), g = lane / 4, t = lane % 4; each
// 32-bit register holds two bf16, the lower index in the low half:
//   A (16 x 16)  a0 = (g, 2t..2t+1)  a1 = (g+8, 2t..)  a2 = (g, 2t+8..)  a3 = (g+8, 2t+8..)
//   B (16 x 8)   b0 = (k 2t..2t+1, n g)  b1 = (k 2t+8..2t+9, n g)
//   C (16 x 8)   c0 = (g, 2t)  c1 = (g, 2t+1)  c2 = (g+8, 2t)  c3 = (g+8, 2t+1)
// An 8 x 8 b16 matrix held one row pair per lane ((g, 2t..2t+1)) is what ldmatrix
// loads and what movmatrix transposes.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace snp {

struct Split2 {
    uint32_t hi, lo;
};

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }

// (a, b) -> packed bf16 pairs hi = bf16(a, b), lo = bf16((a, b) - hi); LO = false
// skips the correction (lo = 0).
template <bool LO>
__device__ __forceinline__ Split2 split2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    Split2 s;
    s.hi = bf16x2_bits(h);
    if constexpr (LO) {
        const float2 hf = __bfloat1622float2(h);
        s.lo = bf16x2_bits(__floats2bfloat162_rn(a - hf.x, b - hf.y));
    } else {
        s.lo = 0u;
    }
    return s;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// D += A B for one m16n8k16 tile.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Split-precision product D += A B with A = Ah + Al, B = Bh + Bl (correction
// terms first, then the leading product); BLO = false: B is exactly bf16.
template <bool BLO>
__device__ __forceinline__ void mma_split(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                                          uint32_t bh1, uint32_t bl0, uint32_t bl1)
{
    mma16816(d, al, bh0, bh1);
    if constexpr (BLO) mma16816(d, ah, bl0, bl1);
    mma16816(d, ah, bh0, bh1);
}

// Four 8 x 8 b16 matrices; lanes 8m..8m+7 give the row addresses of matrix m.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// Transpose of an 8 x 8 b16 matrix held one row pair per lane.
__device__ __forceinline__ uint32_t movm_trans(uint32_t x)
{
    uint32_t y;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(y) : "r"(x));
    return y;
}

// Sum v[] over the eight lanes that share lane % 4 (lane bits 2..4).  Afterwards
// lane g = lane / 4 holds, in v[0 .. V/8), the sums of the original entries
// v[g V/8 .. (g+1) V/8).
template <int V>
__device__ __forceinline__ void reduce_scatter_rows(float (&v)[V])
{
    static_assert(V % 8 == 0, "reduce_scatter_rows needs a multiple of 8 values");
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int s = 16; s >= 4; s >>= 1) {
        const int half = V * s / 32;
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
}

}  // namespace snp
