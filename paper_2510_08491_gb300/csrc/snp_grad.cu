// snp_grad.cu -- per-primitive gradient post-passes of the backward.
//
// k_project_bwd: the raster backward leaves, per (view, primitive), gradients of
// the projection record (G = diag(1/s) R(q)^T R_wc^T, e = G r_c, mu_z, the
// projected centre U_c, V_c, R_wc^T r_c / m, 1/m, (eye - c)/m, constant colour,
// with mu' = (R_wc^T)^-1 (c - eye) and r_c = mu' / mu'_z); this pass chains them
// through the set-up formulas to the centre, log-scales and quaternion (through its
// normalisation) and sums over views.  The chain rule runs in FP32 (a gradient
// needs ~1e-6 relative accuracy, not the record's float-float set-up); each view's
// contribution is added to float-float accumulators (TwoSum), so the sum over views
// does not lose what one view's terms cancel.
// k_color_post: the colour MLP's first layer is evaluated with the folded bias
// h0 = bc1 + Wc1[:, 3:] feat; this pass distributes dL/dh0 to bc1, Wc1[:, 3:]
// and feat, one warp per primitive (lanes over the hidden units, so that the
// accesses to the primitive's record are contiguous).
#include "snp_common.cuh"
#include "snp_df.cuh"
#include "snp_internal.h"

namespace snp {

__device__ __forceinline__ void acc_add(f2 &a, float x) { a = df_add(a, df_from(x)); }

__global__ void __launch_bounds__(256) k_project_bwd(const float *__restrict__ geom, int64_t n,
                                                     const View *__restrict__ views, int n_views,
                                                     const float *__restrict__ g_view, int rgb_grad,
                                                     float *__restrict__ g_geom)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *Gm = geom + i * 16;
    const float c[3] = {Gm[0], Gm[1], Gm[2]};
    const float s[3] = {expf(Gm[3]), expf(Gm[4]), expf(Gm[5])};
    const float is[3] = {1.0f / s[0], 1.0f / s[1], 1.0f / s[2]};
    const float q[4] = {Gm[6], Gm[7], Gm[8], Gm[9]};
    const float iq = 1.0f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
    const float Rq[3][3] = {{1.0f - 2.0f * (y * y + z * z), 2.0f * (x * y - w * z), 2.0f * (x * z + w * y)},
                            {2.0f * (x * y + w * z), 1.0f - 2.0f * (x * x + z * z), 2.0f * (y * z - w * x)},
                            {2.0f * (x * z - w * y), 2.0f * (y * z + w * x), 1.0f - 2.0f * (x * x + y * y)}};
    int am = 0;
    if (s[1] > s[am]) am = 1;
    if (s[2] > s[am]) am = 2;
    const float inv_m = is[am];
    float Minv[3][3];
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) Minv[a][j] = Rq[j][a] * is[a];

    f2 gc[3], gs[3], gR[3][3], grgb[3];
    for (int a = 0; a < 3; ++a) {
        gc[a] = gs[a] = grgb[a] = df_from(0.0f);
        for (int j = 0; j < 3; ++j) gR[a][j] = df_from(0.0f);
    }
    for (int v = 0; v < n_views; ++v) {
        const float *g = g_view + ((int64_t)v * n + i) * kGvFloats;
        const View &V = views[v];
        float Rw[3][3];
        for (int k = 0; k < 9; ++k) Rw[k / 3][k % 3] = V.R[k];
        const float dc[3] = {c[0] - V.eye[0], c[1] - V.eye[1], c[2] - V.eye[2]};
        float mu[3];  // mu' = (R_wc^T)^-1 (c - eye)
        for (int a = 0; a < 3; ++a)
            mu[a] = V.Rti_hi[3 * a + 0] * dc[0] + V.Rti_hi[3 * a + 1] * dc[1] + V.Rti_hi[3 * a + 2] * dc[2];
        const float imz = 1.0f / mu[2];
        const float rc[3] = {mu[0] * imz, mu[1] * imz, 1.0f};
        float G[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = Minv[a][0] * Rw[b][0] + Minv[a][1] * Rw[b][1] + Minv[a][2] * Rw[b][2];
        // dL/dG: columns 0, 1 from f = G dr, all columns from e = G r_c
        float gG[3][3];
        for (int a = 0; a < 3; ++a) {
            gG[a][0] = g[kGvG + 2 * a + 0] + g[kGvE + a] * rc[0];
            gG[a][1] = g[kGvG + 2 * a + 1] + g[kGvE + a] * rc[1];
            gG[a][2] = g[kGvE + a] * rc[2];
        }
        // dL/dr_c from e = G r_c and a_c = R_wc^T r_c / m; U_c = cx + fx r_c.x, V_c = cy + fy r_c.y
        float grc[3];
        for (int b = 0; b < 3; ++b) {
            float t = 0.0f;
            for (int a = 0; a < 3; ++a) t += G[a][b] * g[kGvE + a] + inv_m * Rw[b][a] * g[kGvAc + a];
            grc[b] = t;
        }
        grc[0] += g[kGvU] * V.fx;
        grc[1] += g[kGvV] * V.fy;
        float ginvm = g[kGvInvM];
        for (int a = 0; a < 3; ++a) {
            const float rwc = Rw[0][a] * rc[0] + Rw[1][a] * rc[1] + Rw[2][a] * rc[2];
            ginvm += g[kGvAc + a] * rwc - g[kGvOcm + a] * dc[a];
        }
        // r_c = mu / mu_z
        const float gmu[3] = {grc[0] * imz, grc[1] * imz, g[kGvMz] - (grc[0] * mu[0] + grc[1] * mu[1]) * imz * imz};
        // mu' = (R_wc^T)^-1 (c - eye);  ocm = (eye - c) / m
        for (int b = 0; b < 3; ++b)
            acc_add(gc[b], V.Rti_hi[0 + b] * gmu[0] + V.Rti_hi[3 + b] * gmu[1] + V.Rti_hi[6 + b] * gmu[2] -
                               inv_m * g[kGvOcm + b]);
        float gsv[3] = {0.0f, 0.0f, 0.0f};
        gsv[am] = -ginvm * inv_m * inv_m;
        // G = Minv R_wc^T;  Minv[a][j] = R_q[j][a] / s_a
        for (int a = 0; a < 3; ++a) {
            for (int j = 0; j < 3; ++j) {
                const float gM = gG[a][0] * Rw[0][j] + gG[a][1] * Rw[1][j] + gG[a][2] * Rw[2][j];
                gsv[a] -= gM * Rq[j][a] * is[a] * is[a];
                acc_add(gR[j][a], gM * is[a]);
            }
            acc_add(gs[a], gsv[a]);
        }
        if (rgb_grad)
            for (int k = 0; k < 3; ++k) acc_add(grgb[k], g[kGvRgb + k]);
    }
    // rotation matrix -> normalised quaternion
    float R9[3][3];
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) R9[a][j] = gR[a][j].hi + gR[a][j].lo;
    float gw = 0, gx = 0, gy = 0, gz = 0;
    gx += -4 * x * (R9[1][1] + R9[2][2]);
    gy += -4 * y * (R9[0][0] + R9[2][2]);
    gz += -4 * z * (R9[0][0] + R9[1][1]);
    gx += 2 * y * R9[0][1]; gy += 2 * x * R9[0][1]; gw -= 2 * z * R9[0][1]; gz -= 2 * w * R9[0][1];
    gx += 2 * z * R9[0][2]; gz += 2 * x * R9[0][2]; gw += 2 * y * R9[0][2]; gy += 2 * w * R9[0][2];
    gx += 2 * y * R9[1][0]; gy += 2 * x * R9[1][0]; gw += 2 * z * R9[1][0]; gz += 2 * w * R9[1][0];
    gy += 2 * z * R9[1][2]; gz += 2 * y * R9[1][2]; gw -= 2 * x * R9[1][2]; gx -= 2 * w * R9[1][2];
    gx += 2 * z * R9[2][0]; gz += 2 * x * R9[2][0]; gw -= 2 * y * R9[2][0]; gy -= 2 * w * R9[2][0];
    gy += 2 * z * R9[2][1]; gz += 2 * y * R9[2][1]; gw += 2 * x * R9[2][1]; gx += 2 * w * R9[2][1];
    const float dot = gw * w + gx * x + gy * y + gz * z;
    float *O = g_geom + i * 16;
    O[0] += gc[0].hi + gc[0].lo;
    O[1] += gc[1].hi + gc[1].lo;
    O[2] += gc[2].hi + gc[2].lo;
    for (int a = 0; a < 3; ++a) O[3 + a] += (gs[a].hi + gs[a].lo) * s[a];
    O[6] += (gw - w * dot) * iq;
    O[7] += (gx - x * dot) * iq;
    O[8] += (gy - y * dot) * iq;
    O[9] += (gz - z * dot) * iq;
    if (rgb_grad) {
        O[10] += grgb[0].hi + grgb[0].lo;
        O[11] += grgb[1].hi + grgb[1].lo;
        O[12] += grgb[2].hi + grgb[2].lo;
    }
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_color_post(const void *__restrict__ net, int64_t n, int n_c, int off_feat,
                                                    int off_Wc1, int off_bc1, int stride,
                                                    const float *__restrict__ g_h0, float *__restrict__ g_net)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int64_t base = i * stride;
    float f[kFeat], gf[kFeat];
#pragma unroll
    for (int k = 0; k < kFeat; ++k) {
        f[k] = ld_w<BF16>(net, base + off_feat + k);
        gf[k] = 0.0f;
    }
    for (int j = lane; j < n_c; j += 32) {
        const float g = g_h0[i * n_c + j];
        if (g == 0.0f) continue;
        g_net[base + off_bc1 + j] += g;
        const int64_t w = base + off_Wc1 + (int64_t)j * (3 + kFeat) + 3;
#pragma unroll
        for (int k = 0; k < kFeat; ++k) {
            g_net[w + k] += g * f[k];
            gf[k] = fmaf(ld_w<BF16>(net, w + k), g, gf[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < kFeat; ++k) gf[k] = warp_sum(gf[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kFeat; ++k) g_net[base + off_feat + k] += gf[k];
    }
}

void launch_project_bwd(const float *geom, int64_t n, const View *views, int n_views, const float *g_view,
                        int rgb_grad, float *g_geom, cudaStream_t st)
{
    if (n <= 0) return;
    k_project_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(geom, n, views, n_views, g_view, rgb_grad, g_geom);
    note_launch();
}

void launch_color_post(const void *net, int bf16, int64_t n, int n_c, int off_feat, int off_Wc1, int off_bc1,
                       int stride, const float *g_h0, float *g_net, cudaStream_t st)
{
    if (n <= 0) return;
    const unsigned g = (unsigned)((n * 32 + 255) / 256);  // one warp per primitive
    if (bf16)
        k_color_post<true><<<g, 256, 0, st>>>(net, n, n_c, off_feat, off_Wc1, off_bc1, stride, g_h0, g_net);
    else
        k_color_post<false><<<g, 256, 0, st>>>(net, n, n_c, off_feat, off_Wc1, off_bc1, stride, g_h0, g_net);
    note_launch();
}

}  // namespace snp
