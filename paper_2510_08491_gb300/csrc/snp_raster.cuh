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

// Ray / ellipsoid closest-approach test in unit-sphere coordinates.
struct Hit {
    float tm, half;  // midpoint and half chord (world units along the unit ray)
    float3 dp;       // Minv d
    float3 p;        // closest point to the centre (unit-sphere coordinates)
    float A, B, iA, h2;
};

__device__ __forceinline__ bool intersect(const float *R, float3 d, Hit &h)
{
    const float4 r0 = reinterpret_cast<const float4 *>(R)[0];
    const float4 r1 = reinterpret_cast<const float4 *>(R)[1];
    const float4 r2 = reinterpret_cast<const float4 *>(R)[2];
    // Minv rows: (r0.x r0.y r0.z) (r0.w r1.x r1.y) (r1.z r1.w r2.x); op = (r2.y r2.z r2.w)
    h.dp.x = fmaf(r0.x, d.x, fmaf(r0.y, d.y, r0.z * d.z));
    h.dp.y = fmaf(r0.w, d.x, fmaf(r1.x, d.y, r1.y * d.z));
    h.dp.z = fmaf(r1.z, d.x, fmaf(r1.w, d.y, r2.x * d.z));
    h.A = fmaf(h.dp.x, h.dp.x, fmaf(h.dp.y, h.dp.y, h.dp.z * h.dp.z));
    h.B = fmaf(r2.y, h.dp.x, fmaf(r2.z, h.dp.y, r2.w * h.dp.z));
    h.iA = __fdividef(1.0f, h.A);
    h.tm = -h.B * h.iA;
    h.p.x = fmaf(h.tm, h.dp.x, r2.y);
    h.p.y = fmaf(h.tm, h.dp.y, r2.z);
    h.p.z = fmaf(h.tm, h.dp.z, r2.w);
    h.h2 = 1.0f - fmaf(h.p.x, h.p.x, fmaf(h.p.y, h.p.y, h.p.z * h.p.z));
    if (!(h.h2 > 0.0f)) return false;
    const float x = h.h2 * h.iA;
    h.half = x * rsqrtf(x);
    return true;
}

// alpha_hat of one (ray, primitive) pair.  FORM 0 (stable):
//   Delta_t [b2 + sum_k w2_k cos(phi_k) sinc(theta_k)], phi_k = w0 (W1_k . u_mid + b1_k),
//   theta_k = w0 (W1_k . d) half / m.   FORM 1 (naive, Eq. 8 literally):
//   sum_k w2_k [sin(a_k t_out + psi_k) - sin(a_k t_in + psi_k)] / a_k + b2 (t_out - t_in),
//   a_k = w0 W1_k . d / m, psi_k = w0 (W1_k . (eye - c) / m + b1_k).
template <int FORM>
__device__ __forceinline__ float integral(const float *R, const float *D, int ns, float3 d, const Hit &h)
{
    const float inv_m = R[kRecInvM];
    const float4 *W = reinterpret_cast<const float4 *>(D);
    const float *w2 = D + 4 * ns;
    float acc = 0.0f;
    if constexpr (FORM == 0) {
        const float tmm = h.tm * inv_m, hm = h.half * inv_m;
        const float3 u = make_float3(fmaf(tmm, d.x, R[kRecOcm + 0]), fmaf(tmm, d.y, R[kRecOcm + 1]),
                                     fmaf(tmm, d.z, R[kRecOcm + 2]));
#pragma unroll 4
        for (int k = 0; k < ns; ++k) {
            const float4 w = W[k];
            const float g = fmaf(w.x, d.x, fmaf(w.y, d.y, w.z * d.z));
            const float ph = fmaf(w.x, u.x, fmaf(w.y, u.y, fmaf(w.z, u.z, w.w)));
            acc = fmaf(w2[k] * __cosf(ph), sincf_fast(g * hm), acc);
        }
        return 2.0f * h.half * (w2[ns] + acc);
    } else {
        const float tin = h.tm - h.half, tout = h.tm + h.half;
        const float ox = R[kRecOcm + 0], oy = R[kRecOcm + 1], oz = R[kRecOcm + 2];
#pragma unroll 4
        for (int k = 0; k < ns; ++k) {
            const float4 w = W[k];
            const float ak = fmaf(w.x, d.x, fmaf(w.y, d.y, w.z * d.z)) * inv_m;
            const float psi = fmaf(w.x, ox, fmaf(w.y, oy, fmaf(w.z, oz, w.w)));
            acc = fmaf(w2[k], __fdividef(__sinf(fmaf(ak, tout, psi)) - __sinf(fmaf(ak, tin, psi)), ak), acc);
        }
        return fmaf(w2[ns], tout - tin, acc);
    }
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

// Entry/exit test only (h^2 > 0), the same arithmetic as intersect().
__device__ __forceinline__ bool hit_test(const float *R, float3 d)
{
    Hit h;
    const float4 r0 = reinterpret_cast<const float4 *>(R)[0];
    const float4 r1 = reinterpret_cast<const float4 *>(R)[1];
    const float4 r2 = reinterpret_cast<const float4 *>(R)[2];
    h.dp.x = fmaf(r0.x, d.x, fmaf(r0.y, d.y, r0.z * d.z));
    h.dp.y = fmaf(r0.w, d.x, fmaf(r1.x, d.y, r1.y * d.z));
    h.dp.z = fmaf(r1.z, d.x, fmaf(r1.w, d.y, r2.x * d.z));
    h.A = fmaf(h.dp.x, h.dp.x, fmaf(h.dp.y, h.dp.y, h.dp.z * h.dp.z));
    h.B = fmaf(r2.y, h.dp.x, fmaf(r2.z, h.dp.y, r2.w * h.dp.z));
    h.iA = __fdividef(1.0f, h.A);
    h.tm = -h.B * h.iA;
    h.p.x = fmaf(h.tm, h.dp.x, r2.y);
    h.p.y = fmaf(h.tm, h.dp.y, r2.z);
    h.p.z = fmaf(h.tm, h.dp.z, r2.w);
    h.h2 = 1.0f - fmaf(h.p.x, h.p.x, fmaf(h.p.y, h.p.y, h.p.z * h.p.z));
    return h.h2 > 0.0f;
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
