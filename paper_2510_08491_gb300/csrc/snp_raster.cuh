// snp_raster.cuh -- per-tile rasterizer pieces shared by the forward and backward
// kernels: shared-memory staging of a chunk of a tile's primitive list, the
// ray/ellipsoid test, the closed-form integral (Sec. 3.2, Eq. 8) and the colour MLP.
//
// Shared-memory entry (floats) for one primitive of the chunk:
//   [0, kRecFloats)     projection record (kRec* offsets)
//   density block       per hidden unit k a float4 (w0 W1_k, w0 b1_k), then w2[N_sigma], b2, pad
//   colour block (MLP)  C1[n_c] float4 (Wc1[j][0..2], h0_j = bc1_j + Wc1[j][3..10] . feat),
//                       W2 as bf16 hi[n_c][n_c + 8] then lo[n_c][n_c + 8] (Wc2 = hi + lo;
//                       lo is not staged for bf16 weights), B2[n_c],
//                       C3[n_c] float4 (Wc3[0..2][j], 0), B3 float4
// The folded first-layer bias h0 uses that the feature part of the colour input is
// constant per primitive; only the direction part varies per pixel.  The hidden
// layer runs on the tensor cores over warp batches of 32 rays (snp_mma.cuh).
#pragma once

#include "snp_common.cuh"
#include "snp_df.cuh"
#include "snp_internal.h"
#include "snp_mma.cuh"
#include "snp_tmem.cuh"

namespace snp {

constexpr int kRasterThreads = 256;
constexpr int kMaxChunk = 256;

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }
__host__ __device__ constexpr int den_stride(int ns) { return 4 * ns + round4(ns + 1); }
// Row stride (bf16 elements) of the staged Wc2: the 8 extra elements move each
// row by 16 bytes of bank offset, so the eight 16-byte rows of one ldmatrix
// read hit distinct banks.
__host__ __device__ constexpr int w2_ld(int nc) { return nc + 8; }
__host__ __device__ constexpr int col_stride(int nc) { return nc == 0 ? 0 : nc * w2_ld(nc) + 9 * nc + 4; }
__host__ __device__ constexpr int entry_stride(int ns, int nc) { return kRecFloats + den_stride(ns) + col_stride(nc); }

// Colour-block offsets (floats, from the start of the colour block).
__host__ __device__ constexpr int cb_C1(int) { return 0; }
__host__ __device__ constexpr int cb_W2(int nc) { return 4 * nc; }
__host__ __device__ constexpr int cb_B2(int nc) { return 4 * nc + nc * w2_ld(nc); }
__host__ __device__ constexpr int cb_C3(int nc) { return 5 * nc + nc * w2_ld(nc); }
__host__ __device__ constexpr int cb_B3(int nc) { return 9 * nc + nc * w2_ld(nc); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Stage `cnt` list entries (global record ids s_gid[0..cnt)) of view offset vn
// into shared memory: the projection record and the primitive's packed network
// block (already in the staged layout, see k_pack_net) as 16-byte asynchronous
// copies.  All threads of the block participate; the caller synchronises.
//
// Without a colour network (NC = 0) an entry is only ~23 pieces, so the pieces of
// all entries are spread over the block as one flat range.  Those kernels also
// carry the time-conditioned scene (a.off_wt >= 0): the view's phase xi W_t,k is
// added to the staged w0 b1_k of every hidden unit -- the time term is constant
// along a ray, a per-(view, primitive) shift of the phase (App. Applications).
// Each thread shifts only pieces it copied itself, which its own
// cp.async.wait_group has completed.  (The colour-MLP kernels keep the
// per-entry loop and never see the shift, so their register allocation is
// unchanged.)
// With BF16 weights the lo half of the staged Wc2 is zero and never read: its
// 16-byte pieces of an entry, [w2lo_first, + w2lo_count), are not copied.
__device__ __forceinline__ int w2lo_first(int ns, int nc)
{
    return (kRecFloats + den_stride(ns) + cb_W2(nc) + nc * w2_ld(nc) / 2) / 4;
}
__host__ __device__ constexpr int w2lo_count(int nc) { return nc * w2_ld(nc) / 8; }

// The copies of stage_chunk for a colour-network kernel, without the wait: the
// caller issues more copies (the colour store's) and waits once for all.
template <int NC, bool BF16>
__device__ __forceinline__ void stage_chunk_issue(float *sm, const uint32_t *s_gid, int cnt, int64_t vn,
                                                  const RasterArgs &a, int es)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr int kRec16 = kRecFloats / 4;
    constexpr int skip = BF16 ? w2lo_count(NC) : 0;
    const int lo0 = w2lo_first(a.n_sigma, NC);
    const int per = es / 4 - skip;
    for (int e = 0; e < cnt; ++e) {
        const int64_t gid = s_gid[e];
        const float *rec = a.rec + gid * kRecFloats;
        const float *net = a.npack + (gid - vn) * a.npack_stride;
        float *dst = sm + e * es;
        for (int c = tid; c < per; c += nt) {
            const int q = (skip > 0 && c >= lo0) ? c + skip : c;
            cp_async16(dst + 4 * q, q < kRec16 ? rec + 4 * q : net + 4 * (q - kRec16));
        }
    }
}

// The copies of stage_chunk without a colour network (one flat range of 16-byte
// pieces over all entries), without the wait.
__device__ __forceinline__ void stage_issue_flat(float *sm, const uint32_t *s_gid, int cnt, int64_t vn,
                                                 const RasterArgs &a, int es)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr int kRec16 = kRecFloats / 4;
    const int per = es / 4;  // 16-byte pieces per entry: record, then the network block
    const int total = cnt * per;
    for (int idx = tid; idx < total; idx += nt) {
        const int e = idx / per, q = idx - e * per;
        const int64_t gid = s_gid[e];
        const float *src = q < kRec16 ? a.rec + gid * kRecFloats + 4 * q
                                      : a.npack + (gid - vn) * a.npack_stride + 4 * (q - kRec16);
        cp_async16(sm + e * es + 4 * q, src);
    }
}

// After the calling thread's stage_issue_flat copies have completed (its own
// cp.async wait): the time-conditioned phase shift of the pieces it copied.
template <bool BF16>
__device__ __forceinline__ void stage_shift_flat(float *sm, const uint32_t *s_gid, int cnt, int64_t vn,
                                                 const RasterArgs &a, int es, float xi)
{
    if (a.off_wt < 0) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    constexpr int kRec16 = kRecFloats / 4;
    const int per = es / 4;
    const int total = cnt * per;
    for (int idx = tid; idx < total; idx += nt) {
        const int e = idx / per, q = idx - e * per - kRec16;
        if (q >= 0 && q < a.n_sigma) {
            float *w = sm + e * es + 4 * (q + kRec16) + 3;
            *w = fmaf(xi, ld_w<BF16>(a.net, (s_gid[e] - vn) * a.stride + a.off_wt + q), *w);
        }
    }
}

template <int NC, bool BF16>
__device__ __forceinline__ void stage_chunk(float *sm, const uint32_t *s_gid, int cnt, int64_t vn,
                                            const RasterArgs &a, int es, float xi)
{
    if constexpr (NC == 0) {
        stage_issue_flat(sm, s_gid, cnt, vn, a, es);
        cp_async_wait_all();
        stage_shift_flat<BF16>(sm, s_gid, cnt, vn, a, es, xi);
    } else {
        stage_chunk_issue<NC, BF16>(sm, s_gid, cnt, vn, a, es);
        cp_async_wait_all();
    }
}

// Network block of primitive p in the staged layout (density block, then the
// colour block), one warp per primitive; written once per forward and copied
// into shared memory for every (tile, primitive) pair.
template <int NC, bool BF16>
__global__ void __launch_bounds__(256) k_pack_net(RasterArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= a.n) return;
    const int ns = a.n_sigma;
    const int64_t base = p * a.stride;
    float *D = a.npack + p * a.npack_stride;
    const int dstr = den_stride(ns);
    for (int idx = lane; idx < dstr; idx += 32) {
        float v = 0.0f;
        if (idx < 4 * ns) {
            const int k = idx >> 2, j = idx & 3;
            v = a.omega0 * (j < 3 ? ld_w<BF16>(a.net, base + a.off_W1 + 3 * k + j) : ld_w<BF16>(a.net, base + a.off_b1 + k));
        } else if (idx < 5 * ns) {
            v = ld_w<BF16>(a.net, base + a.off_w2 + (idx - 4 * ns));
        } else if (idx == 5 * ns) {
            v = ld_w<BF16>(a.net, base + a.off_b2);
        }
        D[idx] = v;
    }
    if constexpr (NC > 0) {
        float *C = D + dstr;
        for (int idx = lane; idx < 4 * NC; idx += 32) {
            const int j = idx >> 2, r = idx & 3;
            const int64_t w = base + a.off_Wc1 + (int64_t)j * (3 + kFeat);
            float v;
            if (r < 3) {
                v = ld_w<BF16>(a.net, w + r);
            } else {
                // h0_j = bc1_j + Wc1[j][3..10] . feat (the per-primitive part of the first layer)
                v = ld_w<BF16>(a.net, base + a.off_bc1 + j);
#pragma unroll
                for (int f = 0; f < kFeat; ++f)
                    v = fmaf(ld_w<BF16>(a.net, w + 3 + f), ld_w<BF16>(a.net, base + a.off_feat + f), v);
            }
            C[cb_C1(NC) + idx] = v;
        }
        // Wc2 rows as bf16 hi / lo pairs, padded to w2_ld(NC) columns (with BF16
        // weights the lo half is zero, and neither staging copies nor the kernels
        // read it: it is not written)
        uint32_t *W = reinterpret_cast<uint32_t *>(C + cb_W2(NC));
        constexpr int rowp = w2_ld(NC) / 2;
        for (int q = lane; q < NC * rowp; q += 32) {
            const int row = q / rowp, k = 2 * (q - row * rowp);
            Split2 sp{0u, 0u};
            if (k < NC) {
                const int64_t w = base + a.off_Wc2 + row * NC + k;
                sp = split2<!BF16>(ld_w<BF16>(a.net, w), ld_w<BF16>(a.net, w + 1));
            }
            W[q] = sp.hi;
            if constexpr (!BF16) W[NC * rowp + q] = sp.lo;
        }
        for (int j = lane; j < NC; j += 32) {
            C[cb_B2(NC) + j] = ld_w<BF16>(a.net, base + a.off_bc2 + j);
            C[cb_C3(NC) + 4 * j + 0] = ld_w<BF16>(a.net, base + a.off_Wc3 + j);
            C[cb_C3(NC) + 4 * j + 1] = ld_w<BF16>(a.net, base + a.off_Wc3 + NC + j);
            C[cb_C3(NC) + 4 * j + 2] = ld_w<BF16>(a.net, base + a.off_Wc3 + 2 * NC + j);
            C[cb_C3(NC) + 4 * j + 3] = 0.0f;
        }
        if (lane < 4) C[cb_B3(NC) + lane] = lane < 3 ? ld_w<BF16>(a.net, base + a.off_bc3 + lane) : 0.0f;
    }
}

// Per-tile camera constants for the pair arithmetic.
struct CamK {
    float ifx, ify;  // 1 / fx, 1 / fy
    float fx, fy;
    float3 r0, r1;   // camera x and y axes in world coordinates (rows 0, 1 of R_wc)
};

__device__ __forceinline__ CamK cam_consts(const View &V)
{
    CamK k;
    k.ifx = 1.0f / V.fx;
    k.ify = 1.0f / V.fy;
    k.fx = V.fx;
    k.fy = V.fy;
    k.r0 = make_float3(V.R[0], V.R[1], V.R[2]);
    k.r1 = make_float3(V.R[3], V.R[4], V.R[5]);
    return k;
}

// Ray / ellipsoid intersection, relative to the ray through the centre.  In
// unit-sphere coordinates the ray is (t - mu_z) e + t dp, dp = e + f, f = G dr
// (t in units of the unnormalised ray g).  Closest approach to the centre:
// |p|^2 = mu_z^2 |e x f|^2 / |dp|^2, so h^2 = 1 - |p|^2 needs no cancellation of
// large terms; t_mid = mu_z + s with s = -mu_z (f . dp) / |dp|^2; half chord
// sqrt(h^2 / |dp|^2).
struct Hit {
    float dx, dy;    // dr = (dx, dy, 0)
    float3 f, dp, w; // f = G dr, dp = e + f, w = e x f
    float A, iA, W2, h2, fdp;
    float s, t, half;
};

// Pairs whose FP32 h^2 lies within kBandH2 of the silhouette are evaluated again
// in float-float arithmetic.  The FP32 h^2 has an absolute error of ~1e-7
// (2e-6 at most in an emulation over thin 1:50 primitives); the chord grows like
// sqrt(h^2), so that is a relative error of ~0.5e-7 / h^2 in the chord and in
// alpha_hat, and up to twice that in their derivatives: ~1e-5 at the edge of the
// band (2e-4 at the worst).  Inside the band the value is exact to a few ulp.
// The hit test only needs the sign, which it takes from the record's quadratic in
// FP32 with a per-pair rounding-error margin (hit_test).
constexpr float kBandH2 = 1e-2f;

// h^2 A of a pixel ray from the record's quadratic in the pixel offset
// (X, Y) = (px + .5 - U_c, py + .5 - V_c), in float-float arithmetic: the
// coefficients and U_c, V_c carry their FP64 values as hi + lo, and
// X = (px + .5 - U_hi) - U_lo is formed exactly by TwoSum.  The terms are of
// the order of A and cancel to h^2 A near the silhouette; their float-float
// error, ~2^-46 A, is what is left.
static __device__ __noinline__ float h2A_df(const float *R, float pxh, float pyh)
{
    const float4 q0 = reinterpret_cast<const float4 *>(R + kRecQ)[0];  // c0h c1h c2h c3h
    const float4 q1 = reinterpret_cast<const float4 *>(R + kRecQ)[1];  // c4h c5h c0l c1l
    const float4 q2 = reinterpret_cast<const float4 *>(R + kRecQ)[2];  // c2l c3l c4l c5l
    const float4 u = reinterpret_cast<const float4 *>(R)[3];           // mz mz2 Uhi Ulo
    const float4 v = reinterpret_cast<const float4 *>(R)[4];           // Vhi Vlo ...
    f2 X = df_two_sum(pxh, -u.z);
    X = df_two_sum(X.hi, __fsub_rn(X.lo, u.w));
    f2 Y = df_two_sum(pyh, -v.x);
    Y = df_two_sum(Y.hi, __fsub_rn(Y.lo, v.y));
    const f2 c0{q0.x, q1.z}, c1{q0.y, q1.w}, c2{q0.z, q2.x}, c3{q0.w, q2.y}, c4{q1.x, q2.z}, c5{q1.y, q2.w};
    const f2 a = df_add(c1, df_add(df_mul(c3, X), df_mul(c4, Y)));
    const f2 b = df_add(c2, df_mul(c5, Y));
    const f2 q = df_add(c0, df_add(df_mul(X, a), df_mul(Y, b)));
    return q.hi + q.lo;
}

__device__ __forceinline__ bool intersect(const float *R, const CamK &ck, const PixRay &ry, Hit &h)
{
    const float4 g0 = reinterpret_cast<const float4 *>(R)[0];  // G00 G01 G02 G10
    const float4 g1 = reinterpret_cast<const float4 *>(R)[1];  // G11 G12 G20 G21
    const float4 g2 = reinterpret_cast<const float4 *>(R)[2];  // G22 ex ey ez
    const float4 g3 = reinterpret_cast<const float4 *>(R)[3];  // mz mz2 Uhi Ulo
    const float4 g4 = reinterpret_cast<const float4 *>(R)[4];  // Vhi Vlo ...
    h.dx = ((ry.pxh - g3.z) - g3.w) * ck.ifx;
    h.dy = ((ry.pyh - g4.x) - g4.y) * ck.ify;
    h.f.x = fmaf(g0.x, h.dx, g0.y * h.dy);
    h.f.y = fmaf(g0.w, h.dx, g1.x * h.dy);
    h.f.z = fmaf(g1.z, h.dx, g1.w * h.dy);
    const float3 e = make_float3(g2.y, g2.z, g2.w);
    h.dp = make_float3(e.x + h.f.x, e.y + h.f.y, e.z + h.f.z);
    h.A = fmaf(h.dp.x, h.dp.x, fmaf(h.dp.y, h.dp.y, h.dp.z * h.dp.z));
    h.iA = __fdividef(1.0f, h.A);
    h.w = make_float3(fmaf(e.y, h.f.z, -e.z * h.f.y), fmaf(e.z, h.f.x, -e.x * h.f.z), fmaf(e.x, h.f.y, -e.y * h.f.x));
    h.W2 = fmaf(h.w.x, h.w.x, fmaf(h.w.y, h.w.y, h.w.z * h.w.z));
    h.h2 = 1.0f - g3.y * h.W2 * h.iA;
    if (fabsf(h.h2) < kBandH2) h.h2 = h2A_df(R, ry.pxh, ry.pyh) * h.iA;
    if (!(h.h2 > 0.0f)) return false;
    h.fdp = fmaf(h.f.x, h.dp.x, fmaf(h.f.y, h.dp.y, h.f.z * h.dp.z));
    h.s = -g3.x * h.fdp * h.iA;
    h.t = g3.x + h.s;
    const float x = h.h2 * h.iA;
    // a chord below ~1e-18 (only reachable through the float-float band) counts as a miss
    if (!(x > 1e-36f)) return false;
    h.half = x * rsqrtf(x);
    return true;
}

// Whether the ray enters the ellipsoid: the sign of h^2 A = |e+f|^2 - mu_z^2 |e x f|^2,
// from the record's quadratic in the pixel offset (X, Y) evaluated in FP32 with
// the coefficients' hi parts.  S bounds the sum of the absolute values of its terms;
// the FP32 result is within ~10 ulp of S of the exact value (coefficient rounding,
// the rounding of X and Y, five fused operations), so where |Q| <= 16 2^-24 S the
// sign is taken from the float-float value instead.  Outside that margin and
// outside intersect()'s float-float band the FP32 signs are certain, so the two
// functions always agree on hit or miss.
__device__ __forceinline__ bool hit_test(const float *R, const CamK &ck, const PixRay &ry)
{
    (void)ck;
    const float4 q0 = reinterpret_cast<const float4 *>(R + kRecQ)[0];  // c0h c1h c2h c3h
    const float4 q1 = reinterpret_cast<const float4 *>(R + kRecQ)[1];  // c4h c5h ..
    const float4 g3 = reinterpret_cast<const float4 *>(R)[3];          // mz mz2 Uhi Ulo
    const float4 g4 = reinterpret_cast<const float4 *>(R)[4];          // Vhi Vlo ..
    const float X = (ry.pxh - g3.z) - g3.w;
    const float Y = (ry.pyh - g4.x) - g4.y;
    const float Q = fmaf(X, fmaf(q0.w, X, fmaf(q1.x, Y, q0.y)), fmaf(Y, fmaf(q1.y, Y, q0.z), q0.x));
    const float ax = fabsf(X), ay = fabsf(Y);
    const float S = fmaf(ax, fmaf(fabsf(q0.w), ax, fmaf(fabsf(q1.x), ay, fabsf(q0.y))),
                         fmaf(ay, fmaf(fabsf(q1.y), ay, fabsf(q0.z)), fabsf(q0.x)));
    if (fabsf(Q) <= 9.5367432e-07f * S) return h2A_df(R, ry.pxh, ry.pyh) > 0.0f;  // 16 * 2^-24
    return Q > 0.0f;
}

// alpha_hat of one (ray, primitive) pair.  With u_mid = s a_c + (t / m) dg,
// dg = dx r0 + dy r1 (world offset of the ray direction), FORM 0 (stable):
//   |g| 2 half [b2 + sum_k w2_k cos(phi_k) sinc(theta_k)], phi_k = w0 (W1_k . u_mid + b1_k),
//   theta_k = w0 (W1_k . g) half / m.   FORM 1 (Eq. 8 literally):
//   |g| [sum_k w2_k (sin(a_k t_out + psi_k) - sin(a_k t_in + psi_k)) / a_k + b2 (t_out - t_in)],
//   a_k = w0 W1_k . g / m, psi_k = w0 (W1_k . (eye - c) / m + b1_k).
template <int FORM>
__device__ __forceinline__ float integral(const float *R, const float *D, int ns, const CamK &ck, const PixRay &ry,
                                          const Hit &h)
{
    const float inv_m = R[kRecInvM];
    const float4 *W = reinterpret_cast<const float4 *>(D);
    const float *w2 = D + 4 * ns;
    float acc = 0.0f;
    if constexpr (FORM == 0) {
        const float tm = h.t * inv_m, hm = h.half * inv_m;
        const float3 dg = make_float3(fmaf(h.dx, ck.r0.x, h.dy * ck.r1.x), fmaf(h.dx, ck.r0.y, h.dy * ck.r1.y),
                                      fmaf(h.dx, ck.r0.z, h.dy * ck.r1.z));
        const float3 u = make_float3(fmaf(h.s, R[kRecAc + 0], tm * dg.x), fmaf(h.s, R[kRecAc + 1], tm * dg.y),
                                     fmaf(h.s, R[kRecAc + 2], tm * dg.z));
#pragma unroll 4
        for (int k = 0; k < ns; ++k) {
            const float4 w = W[k];
            const float g = fmaf(w.x, ry.g.x, fmaf(w.y, ry.g.y, w.z * ry.g.z));
            const float ph = fmaf(w.x, u.x, fmaf(w.y, u.y, fmaf(w.z, u.z, w.w)));
            acc = fmaf(w2[k] * __cosf(ph), sincf_fast(g * hm), acc);
        }
        return 2.0f * h.half * ry.gn * (w2[ns] + acc);
    } else {
        const float tin = h.t - h.half, tout = h.t + h.half;
        const float ox = R[kRecOcm + 0], oy = R[kRecOcm + 1], oz = R[kRecOcm + 2];
#pragma unroll 4
        for (int k = 0; k < ns; ++k) {
            const float4 w = W[k];
            const float ak = fmaf(w.x, ry.g.x, fmaf(w.y, ry.g.y, w.z * ry.g.z)) * inv_m;
            const float psi = fmaf(w.x, ox, fmaf(w.y, oy, fmaf(w.z, oz, w.w)));
            acc = fmaf(w2[k], __fdividef(__sinf(fmaf(ak, tout, psi)) - __sinf(fmaf(ak, tin, psi)), ak), acc);
        }
        return ry.gn * fmaf(w2[ns], tout - tin, acc);
    }
}

__device__ __forceinline__ float3 unit_dir(const PixRay &ry)
{
    const float ig = 1.0f / ry.gn;
    return make_float3(ry.g.x * ig, ry.g.y * ig, ry.g.z * ig);
}

// Per-pixel ray data in shared memory (two float4 per pixel slot).
__device__ __forceinline__ void store_ray(float4 *s_ray, int slot, const PixRay &r)
{
    s_ray[2 * slot] = make_float4(r.pxh, r.pyh, r.gn, 0.0f);
    s_ray[2 * slot + 1] = make_float4(r.g.x, r.g.y, r.g.z, 0.0f);
}

__device__ __forceinline__ PixRay load_ray(const float4 *s_ray, int slot)
{
    const float4 a = s_ray[2 * slot], b = s_ray[2 * slot + 1];
    PixRay r;
    r.pxh = a.x;
    r.pyh = a.y;
    r.gn = a.z;
    r.g = make_float3(b.x, b.y, b.z);
    return r;
}

// ---- colour MLP (Sec. 3.1) over a pass of 16 pixel rays of one primitive, one
// warp.  z1 = relu(Wc1_d d + h0), a2 = Wc2 z1 + bc2, z2 = relu(a2),
// c = sigmoid(Wc3 z2 + bc3).  The rays are the rows of the tensor-core tiles:
// lane (g, t) = (lane / 4, lane % 4) holds rows g and g + 8 of the pass, and
// per-unit values live in accumulator layout: x[nt][i] is row (i < 2 ? g : g + 8),
// unit 8 nt + 2 t + (i & 1).

// The two rows of lane (g, t) in a pass over positions r0 .. r0+15 of an entry's
// composited list (n entries): their pixel slots (0 past the end), validity and
// unit ray directions.
struct PassRows {
    int pix0, pix1;
    bool v0, v1;
    float3 d0, d1;
};

__device__ __forceinline__ PassRows pass_rows(const float4 *s_ray, const uint16_t *list, int r0, int n)
{
    const int g = (threadIdx.x & 31) >> 2;
    PassRows p;
    p.v0 = r0 + g < n;
    p.v1 = r0 + g + 8 < n;
    p.pix0 = p.v0 ? list[r0 + g] : 0;
    p.pix1 = p.v1 ? list[r0 + g + 8] : 0;
    p.d0 = unit_dir(load_ray(s_ray, p.pix0));
    p.d1 = unit_dir(load_ray(s_ray, p.pix1));
    return p;
}

// First layer for the pass rows with directions d0, d1.
template <int NC>
__device__ __forceinline__ void color_layer1(const float4 *C1, float3 d0, float3 d1, float (&z)[NC / 8][4])
{
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int nt = 0; nt < NC / 8; ++nt) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float4 w = C1[8 * nt + 2 * t + j];
            z[nt][j] = fmaxf(fmaf(w.x, d0.x, fmaf(w.y, d0.y, fmaf(w.z, d0.z, w.w))), 0.0f);
            z[nt][2 + j] = fmaxf(fmaf(w.x, d1.x, fmaf(w.y, d1.y, fmaf(w.z, d1.z, w.w))), 0.0f);
        }
    }
}

// Accumulator layout -> split A fragments of the 16 x NC block (k tile kt covers
// units 16 kt .. 16 kt + 15, i.e. accumulator tiles 2 kt and 2 kt + 1).
template <int NC>
__device__ __forceinline__ void acc_to_afrag(const float (&x)[NC / 8][4], uint32_t (&ah)[NC / 16][4],
                                             uint32_t (&al)[NC / 16][4])
{
#pragma unroll
    for (int kt = 0; kt < NC / 16; ++kt) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float *src = x[2 * kt + (q >> 1)] + 2 * (q & 1);
            const Split2 sp = split2<true>(src[0], src[1]);
            ah[kt][q] = sp.hi;
            al[kt][q] = sp.lo;
        }
    }
}

// acc[nt] += Z Wc2^T over the pass rows: B fragments are 8 x 8 blocks of the
// row-major staged Wc2 (rows = output units) read by ldmatrix.
template <int NC, bool BF16>
__device__ __forceinline__ void color_gemm_zw(const uint32_t (&zh)[NC / 16][4], const uint32_t (&zl)[NC / 16][4],
                                              const __nv_bfloat16 *Wh, float (&acc)[NC / 8][4])
{
    const int lane = threadIdx.x & 31;
    const __nv_bfloat16 *Wl = Wh + NC * w2_ld(NC);
#pragma unroll
    for (int nt = 0; nt < NC / 8; ++nt) {
#pragma unroll
        for (int kq = 0; kq < NC / 32; ++kq) {
            const int off = (8 * nt + (lane & 7)) * w2_ld(NC) + 32 * kq + 8 * (lane >> 3);
            uint32_t bh[4], bl[4] = {0u, 0u, 0u, 0u};
            ldsm_x4(bh, Wh + off);
            if constexpr (!BF16) ldsm_x4(bl, Wl + off);
            mma_split<!BF16>(acc[nt], zh[2 * kq], zl[2 * kq], bh[0], bh[1], bl[0], bl[1]);
            mma_split<!BF16>(acc[nt], zh[2 * kq + 1], zl[2 * kq + 1], bh[2], bh[3], bl[2], bl[3]);
        }
    }
}

// gz[nk] += GA Wc2 over the pass rows (GA = dL/da2 as A fragments over the
// output units): B fragments are transposed 8 x 8 blocks of the staged Wc2.
template <int NC, bool BF16>
__device__ __forceinline__ void color_gemm_gw(const uint32_t (&gh)[NC / 16][4], const uint32_t (&gl)[NC / 16][4],
                                              const __nv_bfloat16 *Wh, float (&gz)[NC / 8][4])
{
    const int lane = threadIdx.x & 31, m = lane >> 3;
    const __nv_bfloat16 *Wl = Wh + NC * w2_ld(NC);
#pragma unroll
    for (int kn = 0; kn < NC / 16; ++kn) {
#pragma unroll
        for (int nk = 0; nk < NC / 8; nk += 2) {
            const int off = (16 * kn + 8 * (m & 1) + (lane & 7)) * w2_ld(NC) + 8 * (nk + (m >> 1));
            uint32_t bh[4], bl[4] = {0u, 0u, 0u, 0u};
            ldsm_x4_trans(bh, Wh + off);
            if constexpr (!BF16) ldsm_x4_trans(bl, Wl + off);
            mma_split<!BF16>(gz[nk], gh[kn], gl[kn], bh[0], bh[1], bl[0], bl[1]);
            mma_split<!BF16>(gz[nk + 1], gh[kn], gl[kn], bh[2], bh[3], bl[2], bl[3]);
        }
    }
}

// Unit index of slot m (= 2 nt + j) of lane column t in accumulator layout.
__device__ __forceinline__ int acc_unit(int m, int t) { return 8 * (m >> 1) + 2 * t + (m & 1); }

// Colour of the composited pairs at positions r0 .. r0+15 of an entry's list
// (n entries; list holds pixel slots).  Channel c of the pair at slot q goes to
// out[q * qs + c * plane].
template <int NC, bool BF16>
__device__ __forceinline__ void warp_color_pass(const float *Cb, const float4 *s_ray, const uint16_t *list, int r0,
                                                int n, float *out, int qs, int plane)
{
    const int lane = threadIdx.x & 31, t = lane & 3;
    const float4 *C1 = reinterpret_cast<const float4 *>(Cb + cb_C1(NC));
    const float *B2 = Cb + cb_B2(NC);
    const float4 *C3 = reinterpret_cast<const float4 *>(Cb + cb_C3(NC));
    const float4 B3 = *reinterpret_cast<const float4 *>(Cb + cb_B3(NC));
    const __nv_bfloat16 *Wh = reinterpret_cast<const __nv_bfloat16 *>(Cb + cb_W2(NC));
    __syncwarp();
    const PassRows pr = pass_rows(s_ray, list, r0, n);
    float z[NC / 8][4];
    color_layer1<NC>(C1, pr.d0, pr.d1, z);
    uint32_t zh[NC / 16][4], zl[NC / 16][4];
    acc_to_afrag<NC>(z, zh, zl);
    float acc[NC / 8][4];
#pragma unroll
    for (int nt = 0; nt < NC / 8; ++nt) {
        const float2 b = *reinterpret_cast<const float2 *>(B2 + 8 * nt + 2 * t);
        acc[nt][0] = acc[nt][2] = b.x;
        acc[nt][1] = acc[nt][3] = b.y;
    }
    color_gemm_zw<NC, BF16>(zh, zl, Wh, acc);
    float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int nt = 0; nt < NC / 8; ++nt) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float4 w = C3[acc_unit(2 * nt + j, t)];
            const float za = fmaxf(acc[nt][j], 0.0f), zb = fmaxf(acc[nt][2 + j], 0.0f);
            c[0] = fmaf(w.x, za, c[0]);
            c[1] = fmaf(w.y, za, c[1]);
            c[2] = fmaf(w.z, za, c[2]);
            c[3] = fmaf(w.x, zb, c[3]);
            c[4] = fmaf(w.y, zb, c[4]);
            c[5] = fmaf(w.z, zb, c[5]);
        }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        c[q] += __shfl_xor_sync(0xffffffffu, c[q], 1);
        c[q] += __shfl_xor_sync(0xffffffffu, c[q], 2);
    }
    const bool v = t == 0 ? pr.v0 : pr.v1;
    if (t < 2 && v) {
        const int q = (t == 0 ? pr.pix0 : pr.pix1) * qs, o = 3 * t;
        out[q] = sigmoidf_fast(c[o + 0] + B3.x);
        out[plane + q] = sigmoidf_fast(c[o + 1] + B3.y);
        out[2 * plane + q] = sigmoidf_fast(c[o + 2] + B3.z);
    }
}

// Backward of the colour MLP for the composited pairs at positions r0 .. r0+15 of
// an entry's list (n pairs in all).  Per pair: dL/dc = w dL (w: compositing weight at w_e[slot],
// dL: dl[c * npix + slot]) and dL/da3 = dL/dc c (1 - c) (c at col_e[slot * qs +
// c * plane]).  Accumulates, with shared-memory atomics, in the network record layout:
//   WC1 [NC][11]  dL/dWc1 for the direction columns 0..2;   H0 [NC] dL/dh0;
//   AW2 [NC * NC] dL/dWc2 in mma fragment order (element i of lane l of output
//                 tile (mn, nk), i.e. row 16 mn + l/4 + 8 (i >> 1), column
//                 8 nk + 2 (l % 4) + (i & 1), at ((mn NC/8 + nk) 4 + i) 32 + l);
//   W3 [3][NC]    dL/dWc3;  BC2 [NC] dL/dbc2;  AB3 [3] dL/dbc3.
// a2 = Wc2 z1, dL/dz1 = Wc2^T dL/da2 and dL/dWc2 = sum_rays dL/da2 z1^T run on
// the tensor cores; the last takes movmatrix transposes of the pass's register
// fragments, with the 16 rays as the reduction dimension.  With TM (N_c = 32, 64)
// dL/dWc2 is not added to AW2: tcgen05.mma accumulates it in the entry's TMEM
// accumulator (tp.d_tmem) over all of the entry's passes, and the chunk's end reads
// it from there.  ncommit counts this warp's committed MMA groups.
template <int NC, bool BF16, bool TM>
__device__ __forceinline__ void warp_color_bwd_pass(const float *Cb, const float4 *s_ray, const uint16_t *list,
                                                    int r0, int n, const float *w_e, const float *dl, int npix,
                                                    const float *col_e, int qs, int plane, float *WC1, float *H0,
                                                    float *AW2, float *W3, float *BC2, float *AB3,
                                                    const TmemPass &tp, int &ncommit)
{
    static_assert(!TM || NC == 32 || NC == 64, "the TMEM accumulation is built for N_c = 32 and 64");
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float4 *C1 = reinterpret_cast<const float4 *>(Cb + cb_C1(NC));
    const float *B2 = Cb + cb_B2(NC);
    const float4 *C3 = reinterpret_cast<const float4 *>(Cb + cb_C3(NC));
    const __nv_bfloat16 *Wh = reinterpret_cast<const __nv_bfloat16 *>(Cb + cb_W2(NC));
    __syncwarp();
    const PassRows pr = pass_rows(s_ray, list, r0, n);
    const float3 d0 = pr.d0, d1 = pr.d1;
    auto ga3 = [&](bool v, int q) {
        if (!v) return make_float3(0.f, 0.f, 0.f);
        const float w = w_e[q];
        const float cx = col_e[q * qs], cy = col_e[plane + q * qs], cz = col_e[2 * plane + q * qs];
        return make_float3(w * dl[q] * cx * (1.0f - cx), w * dl[npix + q] * cy * (1.0f - cy),
                           w * dl[2 * npix + q] * cz * (1.0f - cz));
    };
    const float3 e0 = ga3(pr.v0, pr.pix0), e1 = ga3(pr.v1, pr.pix1);
    // dL/dbc3 = sum of dL/da3 over the pass.  The four lanes of a row pair hold the
    // same e0, e1: lane (g, t < 3) takes channel t and the sum runs over g only
    // (lane bits 2..4), leaving channel t's total in lane t.
    {
        float b = t == 0 ? e0.x + e1.x : (t == 1 ? e0.y + e1.y : (t == 2 ? e0.z + e1.z : 0.0f));
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (lane < 3 && b != 0.0f) atomicAdd(AB3 + lane, b);
    }
    float z[NC / 8][4];
    color_layer1<NC>(C1, d0, d1, z);
    uint32_t zh[NC / 16][4], zl[NC / 16][4];
    acc_to_afrag<NC>(z, zh, zl);
    float acc[NC / 8][4];
#pragma unroll
    for (int nt = 0; nt < NC / 8; ++nt) {
        const float2 b = *reinterpret_cast<const float2 *>(B2 + 8 * nt + 2 * t);
        acc[nt][0] = acc[nt][2] = b.x;
        acc[nt][1] = acc[nt][3] = b.y;
    }
    color_gemm_zw<NC, BF16>(zh, zl, Wh, acc);
    // dL/dz2 = Wc3^T dL/da3, dL/da2 (ReLU), and the (Wc3, bc2) partials of the two rows
    {
        float pw[NC];
#pragma unroll
        for (int nt = 0; nt < NC / 8; ++nt) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int m = 2 * nt + j;
                const float4 w = C3[acc_unit(m, t)];
                const float a = acc[nt][j], b = acc[nt][2 + j];
                const float za = fmaxf(a, 0.0f), zb = fmaxf(b, 0.0f);
                const float ga = a > 0.0f ? fmaf(w.x, e0.x, fmaf(w.y, e0.y, w.z * e0.z)) : 0.0f;
                const float gb = b > 0.0f ? fmaf(w.x, e1.x, fmaf(w.y, e1.y, w.z * e1.z)) : 0.0f;
                pw[4 * m + 0] = fmaf(e0.x, za, e1.x * zb);
                pw[4 * m + 1] = fmaf(e0.y, za, e1.y * zb);
                pw[4 * m + 2] = fmaf(e0.z, za, e1.z * zb);
                pw[4 * m + 3] = ga + gb;
                acc[nt][j] = ga;
                acc[nt][2 + j] = gb;
            }
        }
        reduce_scatter_rows<NC>(pw);
#pragma unroll
        for (int i = 0; i < NC / 8; ++i) {
            const int idx = g * (NC / 8) + i;
            const int n = acc_unit(idx >> 2, t), c = idx & 3;
            if (pw[i] != 0.0f) atomicAdd(c < 3 ? W3 + c * NC + n : BC2 + n, pw[i]);
        }
    }
    uint32_t gh[NC / 16][4], gl[NC / 16][4];
    acc_to_afrag<NC>(acc, gh, gl);
    // dL/dz1 = Wc2^T dL/da2, dL/da1 (ReLU) and the (Wc1_d, h0) partials
    {
        float gz[NC / 8][4];
#pragma unroll
        for (int nk = 0; nk < NC / 8; ++nk) gz[nk][0] = gz[nk][1] = gz[nk][2] = gz[nk][3] = 0.0f;
        color_gemm_gw<NC, BF16>(gh, gl, Wh, gz);
        float pc[NC];
#pragma unroll
        for (int nk = 0; nk < NC / 8; ++nk) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int m = 2 * nk + j;
                const float ga = z[nk][j] > 0.0f ? gz[nk][j] : 0.0f;
                const float gb = z[nk][2 + j] > 0.0f ? gz[nk][2 + j] : 0.0f;
                pc[4 * m + 0] = fmaf(ga, d0.x, gb * d1.x);
                pc[4 * m + 1] = fmaf(ga, d0.y, gb * d1.y);
                pc[4 * m + 2] = fmaf(ga, d0.z, gb * d1.z);
                pc[4 * m + 3] = ga + gb;
            }
        }
        reduce_scatter_rows<NC>(pc);
#pragma unroll
        for (int i = 0; i < NC / 8; ++i) {
            const int idx = g * (NC / 8) + i;
            const int j = acc_unit(idx >> 2, t), c = idx & 3;
            if (pc[i] != 0.0f) atomicAdd(c < 3 ? WC1 + j * (3 + kFeat) + c : H0 + j, pc[i]);
        }
    }
    // dL/dWc2 += GA^T Z over the pass rows: A = transposed dL/da2 blocks,
    // B = transposed z1 blocks, the 16 rows as the reduction dimension
    uint32_t tzh[NC / 8][2], tzl[NC / 8][2];
#pragma unroll
    for (int nk = 0; nk < NC / 8; ++nk) {
        const int kt = nk >> 1, o = 2 * (nk & 1);
        tzh[nk][0] = movm_trans(zh[kt][o]);
        tzh[nk][1] = movm_trans(zh[kt][o + 1]);
        tzl[nk][0] = movm_trans(zl[kt][o]);
        tzl[nk][1] = movm_trans(zl[kt][o + 1]);
    }
    if constexpr (TM) {
        // The 5th-generation tensor core accumulates the entry's dL/dWc2 in TMEM
        // across all of its passes: this warp writes its pass's operands (A = dL/da2^T,
        // output units x 16 rays; B^T = z1^T, input units x 16 rays; bf16 hi and lo
        // each) to its shared-memory tiles in the K-major core-matrix layout (8-row
        // groups kUmmaSbo apart, the two 8-ray halves kUmmaLbo apart) and lane 0
        // issues the split products.  After the transposes, lane (g, t) holds unit
        // 8 b + g of block b at rays 2t, 2t + 1 (+8 for the second half), one 4-byte
        // pair of the layout.
        //   N_c = 64: A hi at 0, A lo at 2048, B hi at 4096, B lo at 6144 (64 rows
        //             each); D (64 x 64) += A_lo B_hi + A_hi B_lo + A_hi B_hi.
        //   N_c = 32: one 64-row A whose 8-row group 2 b holds the hi half of unit
        //             block b and group 2 b + 1 its lo half (at 0), B hi at 2048, B lo
        //             at 3072 (32 rows each); D (64 x 32) += A B_hi + A B_lo, so that
        //             D row 16 j + r (r < 8) is hi x (hi + lo) of unit 8 j + r and row
        //             16 j + 8 + r is lo x (hi + lo) of the same unit.
        constexpr int kBh = NC == 64 ? 4096 : 2048, kBl = NC == 64 ? 6144 : 3072;
        if (ncommit > 0 && !mbar_wait_bounded(tp.bar, (uint32_t)((ncommit - 1) & 1))) *tp.wait_status = 1;
        char *const st = reinterpret_cast<char *>(tp.stage_ptr);
        const int within = g * 16 + 4 * t;
#pragma unroll
        for (int nk = 0; nk < NC / 8; ++nk) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int off = nk * (int)kUmmaSbo + h * (int)kUmmaLbo + within;
                *reinterpret_cast<uint32_t *>(st + kBh + off) = tzh[nk][h];
                *reinterpret_cast<uint32_t *>(st + kBl + off) = tzl[nk][h];
            }
        }
#pragma unroll
        for (int mn = 0; mn < NC / 16; ++mn) {
            // (unit block, ray half) of th[i]: (2 mn, 0), (2 mn + 1, 0), (2 mn, 1), (2 mn + 1, 1)
            const uint32_t th[4] = {movm_trans(gh[mn][0]), movm_trans(gh[mn][2]), movm_trans(gh[mn][1]),
                                    movm_trans(gh[mn][3])};
            const uint32_t tl[4] = {movm_trans(gl[mn][0]), movm_trans(gl[mn][2]), movm_trans(gl[mn][1]),
                                    movm_trans(gl[mn][3])};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int b = 2 * mn + (i & 1), kh = (i >> 1) * (int)kUmmaLbo + within;
                const int oh = (NC == 64 ? b : 2 * b) * (int)kUmmaSbo + kh;
                const int ol = NC == 64 ? 2048 + oh : oh + (int)kUmmaSbo;
                *reinterpret_cast<uint32_t *>(st + oh) = th[i];
                *reinterpret_cast<uint32_t *>(st + ol) = tl[i];
            }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            // One issuer at a time across the CTA, so that the MMAs of one entry's passes
            // (and its first, overwriting one) reach the tensor core in a defined order.
            int it = 0;
            while (atomicCAS(tp.lock, 0, 1) != 0) {
                if (++it > kWaitLimit) {
                    *tp.wait_status = 1;
                    break;
                }
            }
            __threadfence_block();
            tc_fence_after_sync();
            volatile int *started = tp.started;
            const bool acc_in = *started != 0;
            *started = 1;
            const uint32_t sa = tp.stage;
            constexpr uint32_t idesc = umma_idesc_bf16(64, NC);
            if constexpr (NC == 64) {
                umma_bf16(tp.d_tmem, umma_smem_desc(sa + 2048), umma_smem_desc(sa + kBh), idesc, acc_in);
                umma_bf16(tp.d_tmem, umma_smem_desc(sa), umma_smem_desc(sa + kBl), idesc, true);
                umma_bf16(tp.d_tmem, umma_smem_desc(sa), umma_smem_desc(sa + kBh), idesc, true);
            } else {
                umma_bf16(tp.d_tmem, umma_smem_desc(sa), umma_smem_desc(sa + kBh), idesc, acc_in);
                umma_bf16(tp.d_tmem, umma_smem_desc(sa), umma_smem_desc(sa + kBl), idesc, true);
            }
            umma_commit(tp.bar);
            tc_fence_before_sync();
            __threadfence_block();
            atomicExch(tp.lock, 0);
        }
        __syncwarp();
        ++ncommit;
    } else {
#pragma unroll
        for (int mn = 0; mn < NC / 16; ++mn) {
            const uint32_t th[4] = {movm_trans(gh[mn][0]), movm_trans(gh[mn][2]), movm_trans(gh[mn][1]),
                                    movm_trans(gh[mn][3])};
            const uint32_t tl[4] = {movm_trans(gl[mn][0]), movm_trans(gl[mn][2]), movm_trans(gl[mn][1]),
                                    movm_trans(gl[mn][3])};
#pragma unroll
            for (int nk = 0; nk < NC / 8; ++nk) {
                float d4[4] = {0.f, 0.f, 0.f, 0.f};
                mma16816(d4, tl, tzh[nk][0], tzh[nk][1]);
                mma16816(d4, th, tzl[nk][0], tzl[nk][1]);
                mma16816(d4, th, tzh[nk][0], tzh[nk][1]);
                // fragment order: each atomic of the warp hits 32 consecutive words (no bank conflicts)
                float *dst = AW2 + (mn * (NC / 8) + nk) * 128 + lane;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (d4[i] != 0.0f) atomicAdd(dst + 32 * i, d4[i]);
            }
        }
    }
}

// Rank of pixel slot `slot` among the set bits of a tile's composited mask
// (words[NPIX / 32]): the number of composited pixels with a smaller slot.
template <int NPIX>
__device__ __forceinline__ uint32_t mask_rank(const uint32_t *words, int slot)
{
    uint32_t r = __popc(words[slot >> 5] & ((1u << (slot & 31)) - 1u));
    for (int w = 0; w < (slot >> 5); ++w) r += __popc(words[w]);
    return r;
}

// Warp-aggregated append of `val` to list[] for the lanes with pred set.
__device__ __forceinline__ void list_append(bool pred, uint16_t val, int *count, uint16_t *list)
{
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (m == 0) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(m) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// Exclusive prefix of count[0..n) into pre[0..n] (one warp; n <= 64).
__device__ __forceinline__ void warp_prefix64(const int *count, int n, int *pre)
{
    const unsigned lane = lane_id();
    int a = (int)lane < n ? count[lane] : 0;
    int b = (int)lane + 32 < n ? count[lane + 32] : 0;
    int x = a, y = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int xa = __shfl_up_sync(0xffffffffu, x, o);
        const int yb = __shfl_up_sync(0xffffffffu, y, o);
        if ((int)lane >= o) {
            x += xa;
            y += yb;
        }
    }
    const int tot_a = __shfl_sync(0xffffffffu, x, 31);
    if ((int)lane < n) pre[lane] = x - a;
    if ((int)lane + 32 < n) pre[lane + 32] = tot_a + y - b;
    if (lane == 0) pre[n] = tot_a + __shfl_sync(0xffffffffu, y, 31);
    else __shfl_sync(0xffffffffu, y, 31);
}

// Work items of (1 << sh) pairs per list entry: nb[e] = ceil(count[e] / 2^sh) and
// its exclusive prefix pre[0..n].  One warp.
__device__ __forceinline__ void warp_batch_prefix(const int *count, int n, int sh, int *nb, int *pre)
{
    const unsigned lane = lane_id();
    for (int e = (int)lane; e < n; e += 32) nb[e] = (count[e] + (1 << sh) - 1) >> sh;
    __syncwarp();
    warp_prefix64(nb, n, pre);
}

// Tile shapes: TS x TS pixels, NT threads, PPT pixels per thread.  Warps always
// cover 8 x 4 pixel blocks; pixel slot = k * NT + tid for the thread's k-th pixel.
template <int TS>
struct TileCfg {
    static constexpr int NPIX = TS * TS;
    static constexpr int NT = TS == 8 ? 64 : 256;
    static constexpr int PPT = NPIX / NT;
    static constexpr int MIN_BLOCKS = TS == 8 ? 4 : 2;
};

// CTAs per SM the forward kernel is built for: three (80 registers, a staging
// chunk in a third of the SM's shared memory) at 16-pixel tiles with a colour
// network at most 32 wide, else TileCfg's.
__host__ __device__ constexpr int fwd_min_blocks(int ts, int nc)
{
    return (ts == 16 && nc <= 32) ? 3 : (ts == 8 ? 4 : 2);
}

// CTAs per SM the backward kernel is built for: two (128 registers, a staging
// chunk that fits two CTAs' shared memory) where the colour network is at most
// 32 wide and a thread holds one pixel, else one.
__host__ __device__ constexpr int bwd_min_blocks(int ts, int nc) { return (ts == 16 && nc <= 32) ? 2 : 1; }

template <int TS>
__device__ __forceinline__ void tile_pixel(int tid, int k, int &lx, int &ly)
{
    const int w = tid >> 5, l = tid & 31;
    if constexpr (TS == 8) {
        lx = l & 7;
        ly = w * 4 + (l >> 3);
    } else {
        lx = (w & 1) * 8 + (l & 7) + (TS == 32 ? (k & 1) * 16 : 0);
        ly = (w >> 1) * 4 + (l >> 3) + (TS == 32 ? (k >> 1) * 16 : 0);
    }
}

__device__ __forceinline__ int find_view(const View *views, int n_views, int tile)
{
    int v = 0;
    while (v + 1 < n_views && views[v + 1].tile_off <= tile) ++v;
    return v;
}

}  // namespace snp
