// snp_raster.cuh -- per-tile rasterizer pieces shared by the forward and backward
// kernels: shared-memory staging of a chunk of a tile's primitive list, the
// ray/ellipsoid test, the closed-form integral (Sec. 3.2, Eq. 8) and the colour MLP.
//
// Shared-memory entry (floats) for one primitive of the chunk:
//   [0, 20)             projection record (kRec* offsets)
//   density block       per hidden unit k a float4 (w0 W1_k, w0 b1_k), then w2[N_sigma], b2, pad
//   colour block (MLP)  C1[n_c] float4 (Wc1[j][0..2], h0_j = bc1_j + Wc1[j][3..10] . feat),
//                       W2[n_c][n_c], B2[n_c], C3[n_c] float4 (Wc3[0..2][j], 0), B3 float4
// The folded first-layer bias h0 uses that the feature part of the colour input is
// constant per primitive; only the direction part varies per pixel.
#pragma once

#include "snp_common.cuh"
#include "snp_internal.h"

namespace snp {

constexpr int kRasterThreads = 256;
constexpr int kMaxChunk = 256;

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }
__host__ __device__ constexpr int den_stride(int ns) { return 4 * ns + round4(ns + 1); }
__host__ __device__ constexpr int col_stride(int nc) { return nc == 0 ? 0 : nc * nc + 9 * nc + 4; }
__host__ __device__ constexpr int entry_stride(int ns, int nc) { return kRecFloats + den_stride(ns) + col_stride(nc); }

// Colour-block offsets (floats, from the start of the colour block).
__host__ __device__ constexpr int cb_C1(int) { return 0; }
__host__ __device__ constexpr int cb_W2(int nc) { return 4 * nc; }
__host__ __device__ constexpr int cb_B2(int nc) { return 4 * nc + nc * nc; }
__host__ __device__ constexpr int cb_C3(int nc) { return 5 * nc + nc * nc; }
__host__ __device__ constexpr int cb_B3(int nc) { return 9 * nc + nc * nc; }

// Stage `cnt` list entries (global record ids s_gid[0..cnt)) of view offset vn
// into shared memory.  All threads of the block participate.
template <int NC, bool BF16>
__device__ __forceinline__ void stage_chunk(float *sm, const uint32_t *s_gid, int cnt, int64_t vn,
                                            const RasterArgs &a, int es)
{
    const int ns = a.n_sigma;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int idx = tid; idx < cnt * kRecFloats; idx += nt) {
        const int e = idx / kRecFloats, k = idx - e * kRecFloats;
        sm[e * es + k] = a.rec[(int64_t)s_gid[e] * kRecFloats + k];
    }
    const int dper = 5 * ns + 1;
    for (int idx = tid; idx < cnt * dper; idx += nt) {
        const int e = idx / dper, k = idx - e * dper;
        const int64_t base = ((int64_t)s_gid[e] - vn) * a.stride;
        float *D = sm + e * es + kRecFloats;
        if (k < 3 * ns) {
            const int kk = k / 3, j = k - 3 * kk;
            D[4 * kk + j] = a.omega0 * ld_w<BF16>(a.net, base + a.off_W1 + k);
        } else if (k < 4 * ns) {
            const int kk = k - 3 * ns;
            D[4 * kk + 3] = a.omega0 * ld_w<BF16>(a.net, base + a.off_b1 + kk);
        } else if (k < 5 * ns) {
            const int kk = k - 4 * ns;
            D[4 * ns + kk] = ld_w<BF16>(a.net, base + a.off_w2 + kk);
        } else {
            D[5 * ns] = ld_w<BF16>(a.net, base + a.off_b2);
        }
    }
    if constexpr (NC > 0) {
        const int dstr = den_stride(ns);
        for (int idx = tid; idx < cnt * NC; idx += nt) {
            const int e = idx / NC, j = idx - e * NC;
            const int64_t base = ((int64_t)s_gid[e] - vn) * a.stride;
            float *C = sm + e * es + kRecFloats + dstr;
            const int64_t w = base + a.off_Wc1 + (int64_t)j * (3 + kFeat);
            float h = ld_w<BF16>(a.net, base + a.off_bc1 + j);
#pragma unroll
            for (int f = 0; f < kFeat; ++f)
                h = fmaf(ld_w<BF16>(a.net, w + 3 + f), ld_w<BF16>(a.net, base + a.off_feat + f), h);
            C[4 * j + 0] = ld_w<BF16>(a.net, w + 0);
            C[4 * j + 1] = ld_w<BF16>(a.net, w + 1);
            C[4 * j + 2] = ld_w<BF16>(a.net, w + 2);
            C[4 * j + 3] = h;
            C[cb_B2(NC) + j] = ld_w<BF16>(a.net, base + a.off_bc2 + j);
            C[cb_C3(NC) + 4 * j + 0] = ld_w<BF16>(a.net, base + a.off_Wc3 + j);
            C[cb_C3(NC) + 4 * j + 1] = ld_w<BF16>(a.net, base + a.off_Wc3 + NC + j);
            C[cb_C3(NC) + 4 * j + 2] = ld_w<BF16>(a.net, base + a.off_Wc3 + 2 * NC + j);
            C[cb_C3(NC) + 4 * j + 3] = 0.0f;
            if (j < 4) C[cb_B3(NC) + j] = j < 3 ? ld_w<BF16>(a.net, base + a.off_bc3 + j) : 0.0f;
        }
        for (int idx = tid; idx < cnt * NC * NC; idx += nt) {
            const int e = idx / (NC * NC), k = idx - e * (NC * NC);
            const int64_t base = ((int64_t)s_gid[e] - vn) * a.stride;
            sm[e * es + kRecFloats + dstr + cb_W2(NC) + k] = ld_w<BF16>(a.net, base + a.off_Wc2 + k);
        }
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

// Pairs whose FP32 h^2 lies within this distance of the silhouette are evaluated
// again in FP64 (the chord length grows like sqrt(h^2), so an FP32 error of ~1e-7
// in h^2 would move alpha_hat by ~1e-3 at a grazing ray).
constexpr float kRefineH2 = 1e-4f;

static __device__ __noinline__ void intersect_fp64(const float *R, const CamK &ck, const PixRay &ry, Hit &h)
{
    double G0[3], G1[3], e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        G0[a] = (double)R[kRecG + 3 * a + 0] + (double)R[kRecGlo + 3 * a + 0];
        G1[a] = (double)R[kRecG + 3 * a + 1] + (double)R[kRecGlo + 3 * a + 1];
        e[a] = (double)R[kRecE + a] + (double)R[kRecElo + a];
    }
    const double mz = (double)R[kRecMz] + (double)R[kRecMzlo];
    const double uc = (double)R[kRecU + 0] + (double)R[kRecU + 1];
    const double vc = (double)R[kRecU + 2] + (double)R[kRecU + 3];
    const double dx = ((double)ry.pxh - uc) / (double)ck.fx;
    const double dy = ((double)ry.pyh - vc) / (double)ck.fy;
    double f[3], dp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[a] = G0[a] * dx + G1[a] * dy;
        dp[a] = e[a] + f[a];
    }
    const double A = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
    const double w[3] = {e[1] * f[2] - e[2] * f[1], e[2] * f[0] - e[0] * f[2], e[0] * f[1] - e[1] * f[0]};
    const double W2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double h2 = 1.0 - mz * mz * W2 / A;
    const double fdp = f[0] * dp[0] + f[1] * dp[1] + f[2] * dp[2];
    const double sd = -mz * fdp / A;
    h.dx = (float)dx;
    h.dy = (float)dy;
    h.f = make_float3((float)f[0], (float)f[1], (float)f[2]);
    h.dp = make_float3((float)dp[0], (float)dp[1], (float)dp[2]);
    h.w = make_float3((float)w[0], (float)w[1], (float)w[2]);
    h.A = (float)A;
    h.iA = (float)(1.0 / A);
    h.W2 = (float)W2;
    h.h2 = (float)h2;
    h.fdp = (float)fdp;
    h.s = (float)sd;
    h.t = (float)(mz + sd);
    h.half = (float)sqrt(h2 > 0.0 ? h2 / A : 0.0);
    if (!(h2 > 0.0)) h.h2 = 0.0f;
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
    if (fabsf(h.h2) < kRefineH2) {
        intersect_fp64(R, ck, ry, h);
        return h.h2 > 0.0f && h.half > 0.0f;
    }
    if (!(h.h2 > 0.0f)) return false;
    h.fdp = fmaf(h.f.x, h.dp.x, fmaf(h.f.y, h.dp.y, h.f.z * h.dp.z));
    h.s = -g3.x * h.fdp * h.iA;
    h.t = g3.x + h.s;
    const float x = h.h2 * h.iA;
    h.half = x * rsqrtf(x);
    return true;
}

__device__ __forceinline__ bool hit_test(const float *R, const CamK &ck, const PixRay &ry)
{
    Hit h;
    return intersect(R, ck, ry, h);
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

// Colour MLP of one pixel ray: z1 = relu(Wc1_d d + h0), z2 = relu(Wc2 z1 + bc2),
// c = sigmoid(Wc3 z2 + bc3).  Optionally keeps z1 / z2 for the backward pass.
template <int NC>
__device__ __forceinline__ float3 mlp_color(const float *C, float3 d, float *z1_out = nullptr,
                                            float *z2_out = nullptr)
{
    const float4 *C1 = reinterpret_cast<const float4 *>(C + cb_C1(NC));
    const float *W2 = C + cb_W2(NC);
    const float *B2 = C + cb_B2(NC);
    const float4 *C3 = reinterpret_cast<const float4 *>(C + cb_C3(NC));
    const float4 B3 = *reinterpret_cast<const float4 *>(C + cb_B3(NC));
    float z1[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const float4 w = C1[j];
        z1[j] = fmaxf(fmaf(w.x, d.x, fmaf(w.y, d.y, fmaf(w.z, d.z, w.w))), 0.0f);
        if (z1_out) z1_out[j] = z1[j];
    }
    float c0 = B3.x, c1 = B3.y, c2 = B3.z;
#pragma unroll 1
    for (int j = 0; j < NC; j += 2) {
        const float4 *ra = reinterpret_cast<const float4 *>(W2 + j * NC);
        const float4 *rb = reinterpret_cast<const float4 *>(W2 + (j + 1) * NC);
        float a0 = B2[j], a1 = B2[j + 1];
#pragma unroll
        for (int k = 0; k < NC / 4; ++k) {
            const float4 wa = ra[k], wb = rb[k];
            a0 = fmaf(wa.x, z1[4 * k + 0], a0);
            a1 = fmaf(wb.x, z1[4 * k + 0], a1);
            a0 = fmaf(wa.y, z1[4 * k + 1], a0);
            a1 = fmaf(wb.y, z1[4 * k + 1], a1);
            a0 = fmaf(wa.z, z1[4 * k + 2], a0);
            a1 = fmaf(wb.z, z1[4 * k + 2], a1);
            a0 = fmaf(wa.w, z1[4 * k + 3], a0);
            a1 = fmaf(wb.w, z1[4 * k + 3], a1);
        }
        a0 = fmaxf(a0, 0.0f);
        a1 = fmaxf(a1, 0.0f);
        if (z2_out) {
            z2_out[j] = a0;
            z2_out[j + 1] = a1;
        }
        const float4 wa = C3[j], wb = C3[j + 1];
        c0 = fmaf(wa.x, a0, fmaf(wb.x, a1, c0));
        c1 = fmaf(wa.y, a0, fmaf(wb.y, a1, c1));
        c2 = fmaf(wa.z, a0, fmaf(wb.z, a1, c2));
    }
    return make_float3(sigmoidf_fast(c0), sigmoidf_fast(c1), sigmoidf_fast(c2));
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

// Tile shapes: TS x TS pixels, NT threads, PPT pixels per thread.  Warps always
// cover 8 x 4 pixel blocks; pixel slot = k * NT + tid for the thread's k-th pixel.
template <int TS>
struct TileCfg {
    static constexpr int NPIX = TS * TS;
    static constexpr int NT = TS == 8 ? 64 : 256;
    static constexpr int PPT = NPIX / NT;
    static constexpr int MIN_BLOCKS = TS == 8 ? 4 : 2;
};

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
