// snp_common.cuh -- device-side definitions shared by the libsnp kernels.
//
// Layouts (all device memory):
//   geom   float [n][16]   centre(3) log-scale(3) quaternion wxyz(4) rgb(3) unused(3)
//   net    [n][stride]     weight dtype, field offsets from snp_get_net_layout
//   rec    float [V*n][48] per (view, primitive) projection record (kRec* below)
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

// Projection record (float offsets), per (view, primitive).  The ray of a pixel is
// written relative to the ray through the primitive's centre: with camera-frame
// centre mu, r_c = mu / mu_z and the unnormalised camera-frame pixel ray
// r = ((px+.5-cx)/fx, (py+.5-cy)/fy, 1) = r_c + dr, dr = ((px+.5-U_c)/fx, (py+.5-V_c)/fy, 0)
// where (U_c, V_c) is the projected centre; the line in unit-sphere coordinates is
// (t - mu_z) e + t (e + f) with e = G r_c, f = G dr, G = diag(1/s) R_q^T R_wc^T.
constexpr int kRecG = 0;      // 9: G, row-major
constexpr int kRecE = 9;      // 3: e = G r_c
constexpr int kRecMz = 12;    // 1: mu_z
constexpr int kRecMz2 = 13;   // 1: mu_z^2
constexpr int kRecU = 14;     // 4: U_c hi, U_c lo, V_c hi, V_c lo (FP64 value split into two floats)
constexpr int kRecAc = 18;    // 3: R_wc^T r_c / m,  m = max(s)
constexpr int kRecInvM = 21;  // 1: 1 / m
constexpr int kRecOcm = 22;   // 3: (eye - c) / m  (literal Eq. 8 phases only)
constexpr int kRecRgb = 25;   // 3: constant colour
constexpr int kRecDepth = 28; // 1: camera-frame z of the centre (FP32 key value)
// 12: h^2 A = |e + f|^2 - mu_z^2 |e x f|^2 as a quadratic in the pixel offset
// (X, Y) = (px + .5 - U_c, py + .5 - V_c):  c0 + c1 X + c2 Y + c3 X^2 + c4 X Y + c5 Y^2,
// each coefficient an FP64 value split into float hi + lo, stored as
// [c0h c1h c2h c3h] [c4h c5h c0l c1l] [c2l c3l c4l c5l]
constexpr int kRecQ = 32;
constexpr int kRecFloats = 48;

// Per (view, primitive) gradient record (floats): d/dG columns 0 and 1 (6, row-major
// [3][2]), d/de (3), d/dmu_z (1), d/dU_c (1), d/dV_c (1), d/d(R_wc^T r_c / m) (3),
// d/d(1/m) (1), d/docm (3), d/drgb (3), unused (2).
constexpr int kGvFloats = 24;
constexpr int kGvG = 0, kGvE = 6, kGvMz = 9, kGvU = 10, kGvV = 11, kGvAc = 12, kGvInvM = 15, kGvOcm = 16,
              kGvRgb = 19;

// Per-view constants shared by the kernels.
struct View {
    float R[9];
    float eye[3];
    float fx, fy, cx, cy, z_near;
    int32_t width, height;
    int32_t tiles_x, tiles_y;
    int32_t tile_off;  // first global tile id of this view
    float time;        // timestamp xi_t (time-conditioned scenes)
    int64_t pix_off;   // first pixel of this view in the concatenated image
    // Inverse of R_wc^T (computed on the host in FP64): the stored FP32 rotation is
    // not exactly orthonormal, so the camera-frame centre used for the ray geometry
    // is mu' = (R_wc^T)^-1 (c - eye), for which c - eye = R_wc^T mu' holds exactly.
    // Also as float hi + lo pairs for the float-float record set-up.
    double Rti[9];
    float Rti_hi[9], Rti_lo[9];
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

// Per-pixel ray data: pixel-centre coordinates (exact in FP32) and the
// unnormalised world direction g = R_wc^T ((px+.5-cx)/fx, (py+.5-cy)/fy, 1) with
// its length, in FP32 (px + .5 - cx is exact; a few ulp on g and |g|).
struct PixRay {
    float pxh, pyh, gn;
    float3 g;
};

__device__ __forceinline__ PixRay pixel_ray(const View &v, int px, int py)
{
    PixRay r;
    r.pxh = (float)px + 0.5f;
    r.pyh = (float)py + 0.5f;
    const float x = __fdiv_rn(r.pxh - v.cx, v.fx);
    const float y = __fdiv_rn(r.pyh - v.cy, v.fy);
    r.g = make_float3(fmaf(v.R[0], x, fmaf(v.R[3], y, v.R[6])), fmaf(v.R[1], x, fmaf(v.R[4], y, v.R[7])),
                      fmaf(v.R[2], x, fmaf(v.R[5], y, v.R[8])));
    r.gn = __fsqrt_rn(fmaf(r.g.x, r.g.x, fmaf(r.g.y, r.g.y, r.g.z * r.g.z)));
    return r;
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

// sinc(t) = sin(t) / t and its derivative sinc'(t) = (t cos t - sin t) / t^2.
// Below |t| < kSincSeries both come from their Maclaurin series: sinc =
// sum_n (-1)^n t^2n / (2n+1)!, kept to t^10 (remainder < 3e-11 at |t| = 0.5), and
// sinc' = sum_n (-1)^n 2n t^(2n-1) / (2n+1)!, kept to t^9 (remainder < 1e-12).
// Above it sin and cos come from the MUFU unit (absolute error ~4e-7).  The
// numerator of sinc' cancels to ~t^3 / 3 for small t, so the MUFU form would lose
// up to 1% of sinc' near |t| = 0.05; from 0.5 on the numerator is >= 0.04 and its
// relative error stays near 1e-5.
constexpr float kSincSeries = 0.5f;

__device__ __forceinline__ float sinc_series(float t2)
{
    float p = fmaf(t2, -1.0f / 39916800.0f, 1.0f / 362880.0f);
    p = fmaf(t2, p, -1.0f / 5040.0f);
    p = fmaf(t2, p, 1.0f / 120.0f);
    p = fmaf(t2, p, -1.0f / 6.0f);
    return fmaf(t2, p, 1.0f);
}

__device__ __forceinline__ float sinc_deriv_series(float t, float t2)
{
    float p = fmaf(t2, -1.0f / 3991680.0f, 1.0f / 45360.0f);
    p = fmaf(t2, p, -1.0f / 840.0f);
    p = fmaf(t2, p, 1.0f / 30.0f);
    p = fmaf(t2, p, -1.0f / 3.0f);
    return t * p;
}

__device__ __forceinline__ float sincf_fast(float t)
{
    const float series = sinc_series(t * t);
    const float big = __fdividef(__sinf(t), t);
    return fabsf(t) < kSincSeries ? series : big;
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
