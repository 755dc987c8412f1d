// snp_prep.cu -- preprocessing stages of the tile rasterizer ("preprocessing,
// primitive sorting/tiling" of App. A): per (view, primitive) projection and
// bounding, exclusive scan of tile counts, tile-key emission, a stable LSD radix
// sort of the keys and the per-tile ranges.
//
// Key path: visibility, the pixel rectangle of the silhouette and the depth key
// are evaluated in binary32 with correctly rounded +, -, *, /, sqrt in a fixed,
// written-out order (no contraction), so the keys are bit-reproducible from the
// float32 inputs.  The order is:
//   s_j = exp(log_s_j) by Cody-Waite reduction (ln2 split 16-bit head + tail) and
//         the degree-7 Taylor polynomial of e^r in Horner form, scaled by 2^n;
//   q_hat = q * (1 / sqrt(((w w + x x) + y y) + z z));
//   R(q_hat) from the products xx, yy, zz, xy, xz, yz, wx, wy, wz (standard form);
//   V = (R_wc R) diag(s) with each entry ((a0 b0 + a1 b1) + a2 b2) * s_j;
//   Sigma_ab = (V_a0 V_b0 + V_a1 V_b1) + V_a2 V_b2;  mu = R_wc (c - eye);
//   visible iff (mu_z - max s) > z_near;
//   per image axis, the tangent-plane quadratic of the silhouette (see bound_axis);
//   pixel range [ceil(U_min - 0.5 - 1/32), floor(U_max - 0.5 + 1/32)] clamped to the image.
#include <cuda_runtime.h>
#include <stdint.h>

#include "snp_common.cuh"
#include "snp_df.cuh"
#include "snp_internal.h"

namespace snp {

__device__ __forceinline__ float key_exp(float x)
{
    if (x > 80.0f) x = 80.0f;
    if (x < -80.0f) x = -80.0f;
    const float n = rintf(kmul(x, 0x1.715476p+0f));
    float r = ksub(x, kmul(n, 0x1.62e4p-1f));
    r = ksub(r, kmul(n, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;
    p = kadd(0x1.6c16c2p-10f, kmul(r, p));
    p = kadd(0x1.111112p-7f, kmul(r, p));
    p = kadd(0x1.555556p-5f, kmul(r, p));
    p = kadd(0x1.555556p-3f, kmul(r, p));
    p = kadd(0.5f, kmul(r, p));
    p = kadd(1.0f, kmul(r, p));
    p = kadd(1.0f, kmul(r, p));
    const int e = (int)n + 127;
    return kmul(p, __int_as_float(e << 23));
}

// Pixel-centre range along one image axis covered by the silhouette of the
// ellipsoid with camera-frame centre (ma, ., mz) and covariance entries saa,
// saz, szz.  The plane through the eye containing image line U has normal
// (f, 0, cc - U); it is tangent to the ellipsoid when
//   p^2 (mz^2 - szz) + 2 p f (ma mz - saz) + f^2 (ma^2 - saa) = 0,  p = cc - U,
// with quarter discriminant f^2 (mz^2 saa + ma^2 szz - 2 ma mz saz + saz^2 - saa szz).
__device__ __forceinline__ bool bound_axis(float f, float cc, float ma, float mz, float saa, float saz, float szz,
                                           int npx, int &lo, int &hi)
{
    const float mzz = kmul(mz, mz);
    const float a = ksub(mzz, szz);
    const float maz = kmul(ma, mz);
    const float bq = kmul(f, ksub(maz, saz));
    const float t1 = kmul(mzz, saa);
    const float maa = kmul(ma, ma);
    const float t2 = kmul(maa, szz);
    const float t3 = kmul(2.0f, kmul(maz, saz));
    const float t4 = kmul(saz, saz);
    const float t5 = kmul(saa, szz);
    float D = kadd(t1, t2);
    D = ksub(D, t3);
    D = kadd(D, t4);
    D = ksub(D, t5);
    if (!(D > 0.0f)) D = 0.0f;
    const float sq = kmul(f, ksqrt(D));
    const float pmax = kdiv(ksub(sq, bq), a);
    const float pmin = kdiv(ksub(-bq, sq), a);
    const float umin = ksub(cc, pmax);
    const float umax = ksub(cc, pmin);
    float fl = ceilf(ksub(ksub(umin, 0.5f), 0.03125f));
    float fh = floorf(kadd(ksub(umax, 0.5f), 0.03125f));
    const float lim = (float)(npx - 1);
    if (fl < 0.0f) fl = 0.0f;
    if (fh > lim) fh = lim;
    if (!(fl <= fh)) return false;
    lo = (int)fl;
    hi = (int)fh;
    return true;
}

// One thread per (view, primitive): key-path bounding plus the projection record.
__global__ void __launch_bounds__(256) k_project(const float *__restrict__ geom, int64_t n,
                                                 const View *__restrict__ views, int n_views, int ts,
                                                 float *__restrict__ rec, int4 *__restrict__ trect,
                                                 uint32_t *__restrict__ counts)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n * n_views) return;
    const int v = (int)(gid / n);
    const int64_t i = gid - (int64_t)v * n;
    const View &V = views[v];
    const float4 g0 = reinterpret_cast<const float4 *>(geom + i * 16)[0];
    const float4 g1 = reinterpret_cast<const float4 *>(geom + i * 16)[1];
    const float4 g2 = reinterpret_cast<const float4 *>(geom + i * 16)[2];
    const float4 g3 = reinterpret_cast<const float4 *>(geom + i * 16)[3];
    const float c[3] = {g0.x, g0.y, g0.z};
    const float ls[3] = {g0.w, g1.x, g1.y};
    const float q[4] = {g1.z, g1.w, g2.x, g2.y};
    const float rgb[3] = {g2.z, g2.w, g3.x};

    const float s[3] = {key_exp(ls[0]), key_exp(ls[1]), key_exp(ls[2])};
    float qq = kmul(q[0], q[0]);
    qq = kadd(qq, kmul(q[1], q[1]));
    qq = kadd(qq, kmul(q[2], q[2]));
    qq = kadd(qq, kmul(q[3], q[3]));
    const float inv = kdiv(1.0f, ksqrt(qq));
    const float w = kmul(q[0], inv), x = kmul(q[1], inv), y = kmul(q[2], inv), z = kmul(q[3], inv);
    const float xx = kmul(x, x), yy = kmul(y, y), zz = kmul(z, z);
    const float xy = kmul(x, y), xz = kmul(x, z), yz = kmul(y, z);
    const float wx = kmul(w, x), wy = kmul(w, y), wz = kmul(w, z);
    float R[3][3];
    R[0][0] = ksub(1.0f, kmul(2.0f, kadd(yy, zz)));
    R[0][1] = kmul(2.0f, ksub(xy, wz));
    R[0][2] = kmul(2.0f, kadd(xz, wy));
    R[1][0] = kmul(2.0f, kadd(xy, wz));
    R[1][1] = ksub(1.0f, kmul(2.0f, kadd(xx, zz)));
    R[1][2] = kmul(2.0f, ksub(yz, wx));
    R[2][0] = kmul(2.0f, ksub(xz, wy));
    R[2][1] = kmul(2.0f, kadd(yz, wx));
    R[2][2] = ksub(1.0f, kmul(2.0f, kadd(xx, yy)));
    float Vm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float t = kmul(V.R[3 * a + 0], R[0][j]);
            t = kadd(t, kmul(V.R[3 * a + 1], R[1][j]));
            t = kadd(t, kmul(V.R[3 * a + 2], R[2][j]));
            Vm[a][j] = kmul(t, s[j]);
        }
    auto sig = [&](int a, int b) {
        return kadd(kadd(kmul(Vm[a][0], Vm[b][0]), kmul(Vm[a][1], Vm[b][1])), kmul(Vm[a][2], Vm[b][2]));
    };
    const float sxx = sig(0, 0), sxz = sig(0, 2), szz = sig(2, 2), syy = sig(1, 1), syz = sig(1, 2);
    const float dl[3] = {ksub(c[0], V.eye[0]), ksub(c[1], V.eye[1]), ksub(c[2], V.eye[2])};
    float mu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float t = kmul(V.R[3 * a + 0], dl[0]);
        t = kadd(t, kmul(V.R[3 * a + 1], dl[1]));
        t = kadd(t, kmul(V.R[3 * a + 2], dl[2]));
        mu[a] = t;
    }
    float m = s[0] > s[1] ? s[0] : s[1];
    m = m > s[2] ? m : s[2];

    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    bool vis = ksub(mu[2], m) > V.z_near;
    if (vis) vis = bound_axis(V.fx, V.cx, mu[0], mu[2], sxx, sxz, szz, V.width, x0, x1);
    if (vis) vis = bound_axis(V.fy, V.cy, mu[1], mu[2], syy, syz, szz, V.height, y0, y1);

    int4 tr = make_int4(0, 0, -1, -1);
    uint32_t cnt = 0;
    if (vis) {
        tr = make_int4(x0 / ts, y0 / ts, x1 / ts, y1 / ts);
        cnt = (uint32_t)((tr.z - tr.x + 1) * (tr.w - tr.y + 1));
    }
    trect[gid] = tr;
    counts[gid] = cnt;

    // Projection record: evaluated in float-float arithmetic (~2^-47 relative per
    // operation, snp_df.cuh) from the float32 inputs and rounded once; the fields
    // the grazing-ray evaluation needs exactly keep their hi + lo parts.
    float *r = rec + gid * kRecFloats;
    const f2 one = df_from(1.0f);
    const f2 sd[3] = {df_exp(ls[0]), df_exp(ls[1]), df_exp(ls[2])};
    f2 qd = df_two_prod(q[0], q[0]);
    qd = df_add(qd, df_two_prod(q[1], q[1]));
    qd = df_add(qd, df_two_prod(q[2], q[2]));
    qd = df_add(qd, df_two_prod(q[3], q[3]));
    const f2 iqn = df_rsqrt(qd);
    const f2 W = df_mul_f(iqn, q[0]), X = df_mul_f(iqn, q[1]), Y = df_mul_f(iqn, q[2]), Z = df_mul_f(iqn, q[3]);
    const f2 XX = df_mul(X, X), YY = df_mul(Y, Y), ZZ = df_mul(Z, Z);
    const f2 XY = df_mul(X, Y), XZ = df_mul(X, Z), YZ = df_mul(Y, Z);
    const f2 WX = df_mul(W, X), WY = df_mul(W, Y), WZ = df_mul(W, Z);
    auto two = [](f2 a) { return f2{2.0f * a.hi, 2.0f * a.lo}; };
    const f2 Rq[3][3] = {{df_sub(one, two(df_add(YY, ZZ))), two(df_sub(XY, WZ)), two(df_add(XZ, WY))},
                         {two(df_add(XY, WZ)), df_sub(one, two(df_add(XX, ZZ))), two(df_sub(YZ, WX))},
                         {two(df_sub(XZ, WY)), two(df_add(YZ, WX)), df_sub(one, two(df_add(XX, YY)))}};
    int am = 0;  // m = max(s), ties to the lowest axis
    if (sd[1].hi > sd[am].hi || (sd[1].hi == sd[am].hi && sd[1].lo > sd[am].lo)) am = 1;
    if (sd[2].hi > sd[am].hi || (sd[2].hi == sd[am].hi && sd[2].lo > sd[am].lo)) am = 2;
    const float md = sd[am].hi;
    f2 dc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dc[a] = df_two_sum(c[a], -V.eye[a]);  // c - eye, exactly
    f2 mud[3];  // mu' = (R_wc^T)^-1 (c - eye)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f2 acc = df_mul(f2{V.Rti_hi[3 * a + 0], V.Rti_lo[3 * a + 0]}, dc[0]);
        acc = df_add(acc, df_mul(f2{V.Rti_hi[3 * a + 1], V.Rti_lo[3 * a + 1]}, dc[1]));
        mud[a] = df_add(acc, df_mul(f2{V.Rti_hi[3 * a + 2], V.Rti_lo[3 * a + 2]}, dc[2]));
    }
    const f2 rc[2] = {df_div(mud[0], mud[2]), df_div(mud[1], mud[2])};
    // G = diag(1/s) R_q^T R_wc^T:  G[a][b] = sum_j R_q[j][a] R_wc[b][j] / s_a
    f2 G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const f2 is = df_div(one, sd[a]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            f2 t = df_mul_f(Rq[0][a], V.R[3 * b + 0]);
            t = df_add(t, df_mul_f(Rq[1][a], V.R[3 * b + 1]));
            t = df_add(t, df_mul_f(Rq[2][a], V.R[3 * b + 2]));
            G[a][b] = df_mul(t, is);
        }
    }
    f2 e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) r[kRecG + 3 * a + b] = G[a][b].hi;
        e[a] = df_add(df_add(df_mul(G[a][0], rc[0]), df_mul(G[a][1], rc[1])), G[a][2]);
        r[kRecE + a] = e[a].hi;
        // R_wc^T r_c / m
        const float rwc = fmaf(V.R[0 + a], rc[0].hi, fmaf(V.R[3 + a], rc[1].hi, V.R[6 + a]));
        r[kRecAc + a] = rwc / md;
        r[kRecOcm + a] = -(dc[a].hi + dc[a].lo) / md;
        r[kRecRgb + a] = rgb[a];
    }
    const f2 mz = mud[2], mz2 = df_mul(mz, mz);
    r[kRecMz] = mz.hi;
    r[kRecMz2] = mz2.hi;
    // h^2 A = |e + f|^2 - mu_z^2 |e x f|^2 with f = G0 dx + G1 dy (columns 0, 1 of G),
    // dx = X / fx, dy = Y / fy: a quadratic in the pixel offset (X, Y)
    {
        const f2 G0[3] = {G[0][0], G[1][0], G[2][0]}, G1[3] = {G[0][1], G[1][1], G[2][1]};
        auto cross = [](const f2 *u, const f2 *w, f2 *o) {
            o[0] = df_sub(df_mul(u[1], w[2]), df_mul(u[2], w[1]));
            o[1] = df_sub(df_mul(u[2], w[0]), df_mul(u[0], w[2]));
            o[2] = df_sub(df_mul(u[0], w[1]), df_mul(u[1], w[0]));
        };
        auto dot = [](const f2 *u, const f2 *w) {
            return df_add(df_add(df_mul(u[0], w[0]), df_mul(u[1], w[1])), df_mul(u[2], w[2]));
        };
        f2 x0[3], x1[3];
        cross(e, G0, x0);
        cross(e, G1, x1);
        const f2 ifx = df_div(one, df_from(V.fx)), ify = df_div(one, df_from(V.fy));
        const f2 ifxx = df_mul(ifx, ifx), ifyy = df_mul(ify, ify), ifxy = df_mul(ifx, ify);
        const f2 c[6] = {dot(e, e),
                         two(df_mul(dot(e, G0), ifx)),
                         two(df_mul(dot(e, G1), ify)),
                         df_mul(df_sub(dot(G0, G0), df_mul(mz2, dot(x0, x0))), ifxx),
                         two(df_mul(df_sub(dot(G0, G1), df_mul(mz2, dot(x0, x1))), ifxy)),
                         df_mul(df_sub(dot(G1, G1), df_mul(mz2, dot(x1, x1))), ifyy)};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            r[kRecQ + k] = c[k].hi;
            r[kRecQ + 6 + k] = c[k].lo;
        }
    }
    const f2 uc = df_add(df_from(V.cx), df_mul_f(rc[0], V.fx));
    const f2 vc = df_add(df_from(V.cy), df_mul_f(rc[1], V.fy));
    r[kRecU + 0] = uc.hi;
    r[kRecU + 1] = uc.lo;
    r[kRecU + 2] = vc.hi;
    r[kRecU + 3] = vc.lo;
    r[kRecInvM] = 1.0f / md;
    r[kRecDepth] = mu[2];
    r[29] = r[30] = r[31] = 0.0f;
    r[44] = r[45] = r[46] = r[47] = 0.0f;
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (reduce-then-scan, 4096 items per block).
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const unsigned lane = lane_id(), wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        uint32_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (unsigned)o) s += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = s - t;
        if (lane == kScanThreads / 32 - 1) *total = s;
    }
    __syncthreads();
    uint32_t r = x - v + warp_tot[wid];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                              uint32_t *__restrict__ partial)
{
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    s = (uint32_t)warp_sum_u64(s);
    __shared__ uint32_t ws[kScanThreads / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

// Scans one block of items in place into out (exclusive) adding `carry[blockIdx]`.
__global__ void __launch_bounds__(kScanThreads) k_scan_block(const uint32_t *__restrict__ in, int64_t n,
                                                             uint32_t *__restrict__ out,
                                                             const uint32_t *__restrict__ carry,
                                                             uint32_t *__restrict__ total)
{
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    __shared__ uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, &tot);
    const uint32_t c = carry ? carry[blockIdx.x] : 0u;
    pre += c;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
    if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) *total = c + tot;
}

// Recursive exclusive scan: out[i] = sum in[0..i), *total = sum of all (device).
// `tmp` needs scan_temp_words(n) words.
int64_t scan_temp_words(int64_t n)
{
    if (n <= kScanBlock) return 0;
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    return 2 * nb + scan_temp_words(nb) + 64;
}

void scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total, uint32_t *tmp, cudaStream_t st)
{
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return;
    }
    if (n <= kScanBlock) {
        k_scan_block<<<1, kScanThreads, 0, st>>>(in, n, out, nullptr, total);
        note_launch();
        return;
    }
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    uint32_t *partial = tmp;
    uint32_t *carry = tmp + nb;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partial);
    note_launch();
    scan_u32(partial, carry, nb, total, tmp + 2 * nb, st);
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, out, carry, nullptr);
    note_launch();
}

// ---------------------------------------------------------------------------
// Key emission: one thread per (view, primitive), tiles of its rectangle row-major.
__global__ void __launch_bounds__(256) k_emit(const int4 *__restrict__ trect, const uint32_t *__restrict__ counts,
                                              const uint32_t *__restrict__ offsets, const float *__restrict__ rec,
                                              int64_t n, const View *__restrict__ views, int n_views,
                                              uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                              int64_t cap, int32_t *__restrict__ flags)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= n * n_views) return;
    const uint32_t cnt = counts[gid];
    if (cnt == 0) return;
    const int v = (int)(gid / n);
    const View &V = views[v];
    const int4 tr = trect[gid];
    const uint64_t dbits = (uint64_t)__float_as_uint(rec[gid * kRecFloats + kRecDepth]);
    const int64_t base = offsets[gid];
    if (base + cnt > cap) {
        atomicOr(flags, 1);
        return;
    }
    int j = 0;
    for (int ty = tr.y; ty <= tr.w; ++ty)
        for (int tx = tr.x; tx <= tr.z; ++tx, ++j) {
            const uint64_t tile = (uint64_t)(V.tile_off + ty * V.tiles_x + tx);
            keys[base + j] = (tile << 32) | dbits;
            vals[base + j] = (uint32_t)gid;
        }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (u64 key, u32 value), 8-bit digits, 4096 items per
// block.  Each pass: per-block digit histograms (digit-major) -> exclusive scan
// -> stable scatter.  A pass reads the digit (key >> shift) & dmask; the last
// pass masks off the key bits at and above the sorted width.  Inside a block a warp owns 512 consecutive items and walks
// them in strips of 32; the rank of an item is (items of its digit in earlier
// warps) + (in earlier strips of its warp) + (in lower lanes of its strip).
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortBlock = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t *__restrict__ keys,
                                                             const uint32_t *__restrict__ n_ptr, int shift,
                                                             uint32_t dmask, uint32_t *__restrict__ hist,
                                                             int nblocks)
{
    __shared__ uint32_t h[kSortWarps][256];
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = *n_ptr;
    const int wid = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t idx = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[wid][(uint32_t)(keys[idx] >> shift) & dmask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
        hist[(int64_t)d * nblocks + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t *__restrict__ kin,
                                                                const uint32_t *__restrict__ vin,
                                                                uint64_t *__restrict__ kout,
                                                                uint32_t *__restrict__ vout,
                                                                const uint32_t *__restrict__ n_ptr, int shift,
                                                                uint32_t dmask, const uint32_t *__restrict__ offs,
                                                                int nblocks)
{
    __shared__ uint32_t wcnt[kSortWarps][257];
    __shared__ uint32_t gofs[256];
    for (int i = threadIdx.x; i < kSortWarps * 257; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    for (int d = threadIdx.x; d < 256; d += kSortThreads) gofs[d] = offs[(int64_t)d * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t n = *n_ptr;
    const unsigned lane = lane_id();
    const int wid = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)blockIdx.x * kSortBlock + (int64_t)wid * (kSortItems * 32);
    uint64_t k[kSortItems];
    uint32_t v[kSortItems];
    uint32_t rank[kSortItems];
    uint32_t dig[kSortItems];
#pragma unroll
    for (int s = 0; s < kSortItems; ++s) {
        const int64_t idx = wbase + s * 32 + lane;
        const bool ok = idx < n;
        k[s] = ok ? kin[idx] : 0ull;
        v[s] = ok ? vin[idx] : 0u;
        dig[s] = ok ? ((uint32_t)(k[s] >> shift) & dmask) : 256u;
    }
#pragma unroll
    for (int s = 0; s < kSortItems; ++s) {
        const uint32_t d = dig[s];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned lower = peers & ((1u << lane) - 1u);
        const uint32_t before = wcnt[wid][d];
        rank[s] = before + __popc(lower);
        __syncwarp();
        if (lower == 0) wcnt[wid][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for each digit
    for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kSortItems; ++s) {
        const uint32_t d = dig[s];
        if (d < 256u) {
            const uint32_t pos = gofs[d] + wcnt[wid][d] + rank[s];
            kout[pos] = k[s];
            vout[pos] = v[s];
        }
    }
}

int64_t sort_hist_words(int64_t n_bound) { return 256 * ((n_bound + kSortBlock - 1) / kSortBlock); }

// Sorts (keys, vals) by bits [0, nbits) of the key; higher bits do not take part.
// n is on the device (<= n_bound).
// Returns true when the result ended in the *_alt buffers.
bool radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, const uint32_t *d_n,
                int64_t n_bound, int nbits, uint32_t *hist, uint32_t *hist_scan, uint32_t *scan_tmp, cudaStream_t st)
{
    if (n_bound <= 0) return false;
    const int nblocks = (int)((n_bound + kSortBlock - 1) / kSortBlock);
    bool alt = false;
    for (int shift = 0; shift < nbits; shift += 8) {
        const uint64_t *ki = alt ? keys_alt : keys;
        const uint32_t *vi = alt ? vals_alt : vals;
        uint64_t *ko = alt ? keys : keys_alt;
        uint32_t *vo = alt ? vals : vals_alt;
        const uint32_t dmask = nbits - shift >= 8 ? 255u : (1u << (nbits - shift)) - 1u;
        k_radix_hist<<<nblocks, kSortThreads, 0, st>>>(ki, d_n, shift, dmask, hist, nblocks);
        note_launch();
        scan_u32(hist, hist_scan, (int64_t)256 * nblocks, nullptr, scan_tmp, st);
        k_radix_scatter<<<nblocks, kSortThreads, 0, st>>>(ki, vi, ko, vo, d_n, shift, dmask, hist_scan, nblocks);
        note_launch();
        alt = !alt;
    }
    return alt;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tile_ranges(const uint64_t *__restrict__ keys,
                                                     const uint32_t *__restrict__ n_ptr, uint2 *__restrict__ ranges)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = *n_ptr;
    if (i >= n) return;
    const uint32_t t = (uint32_t)(keys[i] >> 32);
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
    if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
}

void launch_project(const float *geom, int64_t n, const View *views, int n_views, int ts, float *rec, int4 *trect,
                    uint32_t *counts, cudaStream_t st)
{
    const int64_t tot = n * n_views;
    if (tot <= 0) return;
    k_project<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(geom, n, views, n_views, ts, rec, trect, counts);
    note_launch();
}

void launch_emit(const int4 *trect, const uint32_t *counts, const uint32_t *offsets, const float *rec, int64_t n,
                 const View *views, int n_views, uint64_t *keys, uint32_t *vals, int64_t cap, int32_t *flags,
                 cudaStream_t st)
{
    const int64_t tot = n * n_views;
    if (tot <= 0) return;
    k_emit<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(trect, counts, offsets, rec, n, views, n_views, keys, vals,
                                                          cap, flags);
    note_launch();
}

// Number of keys the sort and the ranges may touch: the emitted total, clamped to
// the key capacity (an overflow is flagged by k_emit and reported on the host).
__global__ void k_clamp_count(const uint32_t *__restrict__ total, int64_t cap, uint32_t *__restrict__ out)
{
    const uint32_t t = *total;
    *out = (int64_t)t > cap ? (uint32_t)cap : t;
}

void launch_clamp_count(const uint32_t *total, int64_t cap, uint32_t *out, cudaStream_t st)
{
    k_clamp_count<<<1, 1, 0, st>>>(total, cap, out);
    note_launch();
}

void launch_tile_ranges(const uint64_t *keys, const uint32_t *d_n, int64_t n_bound, uint2 *ranges, cudaStream_t st)
{
    if (n_bound <= 0) return;
    k_tile_ranges<<<(unsigned)((n_bound + 255) / 256), 256, 0, st>>>(keys, d_n, ranges);
    note_launch();
}

}  // namespace snp
