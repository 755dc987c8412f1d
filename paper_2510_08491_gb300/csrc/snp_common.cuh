// snp_common.cuh -- device-side definitions shared by the libsnp kernels.
//
// Layouts (all device memory):
//   geom   float [n][16]   centre(3) log-scale(3) quaternion wxyz(4) rgb(3) unused(3)
//   net    [n][stride]     weight dtype, field offsets from snp_get_net_layout
//   rec    float [V*n][20] per (view, primitive) projection record (kRec* below)
//   trect  int4  [V*n]     inclusive tile rectangle tx0, ty0, tx1, ty1
//   keys   u64   [K]       (global tile << 32) | float bits of the camera-frame depth
//   vals   u32   [K]       view * n + primitive
//   ranges uint2 [T]       [start, end) of each tile's run in the sorted keys
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "snp.h"

namespace snp {

constexpr int kFeat = SNP_FEAT_DIM;
constexpr int kMaxViews = 64;

// Projection record (float offsets).
constexpr int kRecMinv = 0;   // 9: diag(1/s) R_q^T, world offset -> unit-sphere coordinates
constexpr int kRecOp = 9;     // 3: Minv (eye - c)
constexpr int kRecOcm = 12;   // 3: (eye - c) / m,  m = max(s)
constexpr int kRecInvM = 15;  // 1: 1 / m
constexpr int kRecRgb = 16;   // 3: constant colour
constexpr int kRecDepth = 19; // 1: camera-frame z of the centre
constexpr int kRecFloats = 20;

// Per (view, primitive) geometry-gradient record (floats): d/dMinv (9), d/dop (3),
// d/docm (3), d/d(1/m) (1), d/drgb (3), unused (1).
constexpr int kGvFloats = 20;

// Per-view constants shared by the kernels.
struct View {
    float R[9];
    float eye[3];
    float fx, fy, cx, cy, z_near;
    int32_t width, height;
    int32_t tiles_x, tiles_y;
    int32_t tile_off;  // first global tile id of this view
    int32_t pad_;
    int64_t pix_off;   // first pixel of this view in the concatenated image
};

// Field offsets of one primitive's network record (elements), see snp_net_layout.
struct NetLayout {
    int32_t W1, b1, w2, b2, feat, Wc1, bc1, Wc2, bc2, Wc3, bc3, stride;
};

// ---------------------------------------------------------------------------
// Correctly rounded binary32 operations for the key path (never contracted).
__device__ __forceinline__ float kmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float kadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ksub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float kdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ksqrt(float a) { return __fsqrt_rn(a); }

// Pixel ray (unit, world frame) through the centre of pixel (px, py), evaluated in
// FP64 once per pixel and rounded to FP32 (the ray position near a primitive far
// from the camera amplifies any error of d by the distance).
__device__ __forceinline__ float3 pixel_ray(const View &v, int px, int py)
{
    const double x = ((double)px + 0.5 - (double)v.cx) / (double)v.fx;
    const double y = ((double)py + 0.5 - (double)v.cy) / (double)v.fy;
    const double rx = (double)v.R[0] * x + (double)v.R[3] * y + (double)v.R[6];
    const double ry = (double)v.R[1] * x + (double)v.R[4] * y + (double)v.R[7];
    const double rz = (double)v.R[2] * x + (double)v.R[5] * y + (double)v.R[8];
    const double inv = 1.0 / sqrt(rx * rx + ry * ry + rz * rz);
    return make_float3((float)(rx * inv), (float)(ry * inv), (float)(rz * inv));
}

template <bool BF16>
__device__ __forceinline__ float ld_w(const void *p, int64_t i)
{
    if constexpr (BF16)
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
    else
        return reinterpret_cast<const float *>(p)[i];
}

__device__ __forceinline__ float sigmoidf_fast(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

// sin(t)/t: Taylor polynomial below |t| < 0.05 (truncation < 4e-12), MUFU sin over t otherwise.
__device__ __forceinline__ float sincf_fast(float t)
{
    float t2 = t * t;
    float poly = fmaf(t2, fmaf(t2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    float big = __fdividef(__sinf(t), t);
    return fabsf(t) < 0.05f ? poly : big;
}

// d/dt sinc(t) = (t cos t - sin t) / t^2; series -t/3 + t^3/30 for small t.
__device__ __forceinline__ float sincf_deriv(float t, float s, float c)
{
    float t2 = t * t;
    float poly = t * fmaf(t2, 1.0f / 30.0f, -1.0f / 3.0f);
    float big = __fdividef(fmaf(t, c, -s), t2);
    return fabsf(t) < 0.05f ? poly : big;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduce-scatter of 32 per-lane values across the warp: on return lane l holds
// the warp-wide sum of v[l].  31 shuffles for 32 sums.
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32])
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            float send = upper ? v[i] : v[i + s];
            float keep = upper ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// Host-side launch helpers implemented in the .cu files.
struct Workspace;

}  // namespace snp
