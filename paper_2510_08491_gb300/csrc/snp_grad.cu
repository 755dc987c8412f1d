// snp_grad.cu -- per-primitive gradient post-passes of the backward.
//
// k_project_bwd: the raster backward leaves, per (view, primitive), gradients of
// the projection record (G = diag(1/s) R(q)^T R_wc^T, e = G r_c, mu_z, the
// projected centre U_c, V_c, R_wc^T r_c / m, 1/m, (eye - c)/m, constant colour,
// with mu' = (R_wc^T)^-1 (c - eye) and r_c = mu' / mu'_z); this pass chains them through
// the FP64 set-up formulas to the centre, log-scales and quaternion (through its
// normalisation) and sums over views.
// k_color_post: the colour MLP's first layer is evaluated with the folded bias
// h0 = bc1 + Wc1[:, 3:] feat; this pass distributes dL/dh0 to bc1, Wc1[:, 3:]
// and feat.
#include "snp_common.cuh"
#include "snp_internal.h"

namespace snp {

__global__ void __launch_bounds__(256) k_project_bwd(const float *__restrict__ geom, int64_t n,
                                                     const View *__restrict__ views, int n_views,
                                                     const float *__restrict__ g_view, int rgb_grad,
                                                     float *__restrict__ g_geom)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *Gm = geom + i * 16;
    const double c[3] = {Gm[0], Gm[1], Gm[2]};
    const double s[3] = {exp((double)Gm[3]), exp((double)Gm[4]), exp((double)Gm[5])};
    const double q[4] = {Gm[6], Gm[7], Gm[8], Gm[9]};
    const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double iq = 1.0 / qn;
    const double w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
    const double Rq[3][3] = {{1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},
                             {2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)},
                             {2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)}};
    int am = 0;
    if (s[1] > s[am]) am = 1;
    if (s[2] > s[am]) am = 2;
    const double m = s[am], inv_m = 1.0 / m;
    double Minv[3][3];
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) Minv[a][j] = Rq[j][a] / s[a];

    double gc[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gR[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, grgb[3] = {0, 0, 0};
    for (int v = 0; v < n_views; ++v) {
        const float *g = g_view + ((int64_t)v * n + i) * kGvFloats;
        const View &V = views[v];
        double Rw[3][3];
        for (int k = 0; k < 9; ++k) Rw[k / 3][k % 3] = V.R[k];
        const double dc[3] = {c[0] - V.eye[0], c[1] - V.eye[1], c[2] - V.eye[2]};
        double mu[3];  // mu' = (R_wc^T)^-1 (c - eye)
        for (int a = 0; a < 3; ++a) mu[a] = V.Rti[3 * a + 0] * dc[0] + V.Rti[3 * a + 1] * dc[1] + V.Rti[3 * a + 2] * dc[2];
        const double rc[3] = {mu[0] / mu[2], mu[1] / mu[2], 1.0};
        double G[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = Minv[a][0] * Rw[b][0] + Minv[a][1] * Rw[b][1] + Minv[a][2] * Rw[b][2];
        // dL/dG: columns 0, 1 from f = G dr, all columns from e = G r_c
        double gG[3][3];
        for (int a = 0; a < 3; ++a) {
            gG[a][0] = g[kGvG + 2 * a + 0] + g[kGvE + a] * rc[0];
            gG[a][1] = g[kGvG + 2 * a + 1] + g[kGvE + a] * rc[1];
            gG[a][2] = g[kGvE + a] * rc[2];
        }
        // dL/dr_c from e = G r_c and a_c = R_wc^T r_c / m; U_c = cx + fx r_c.x, V_c = cy + fy r_c.y
        double grc[3];
        for (int b = 0; b < 3; ++b) {
            double t = 0.0;
            for (int a = 0; a < 3; ++a) t += G[a][b] * g[kGvE + a] + inv_m * Rw[b][a] * g[kGvAc + a];
            grc[b] = t;
        }
        grc[0] += (double)g[kGvU] * V.fx;
        grc[1] += (double)g[kGvV] * V.fy;
        double ginvm = g[kGvInvM];
        for (int a = 0; a < 3; ++a) {
            const double rwc = Rw[0][a] * rc[0] + Rw[1][a] * rc[1] + Rw[2][a] * rc[2];
            ginvm += g[kGvAc + a] * rwc - (double)g[kGvOcm + a] * dc[a];
        }
        // r_c = mu / mu_z
        double gmu[3];
        gmu[0] = grc[0] / mu[2];
        gmu[1] = grc[1] / mu[2];
        gmu[2] = (double)g[kGvMz] - (grc[0] * mu[0] + grc[1] * mu[1]) / (mu[2] * mu[2]);
        // mu' = (R_wc^T)^-1 (c - eye);  ocm = (eye - c) / m
        for (int b = 0; b < 3; ++b)
            gc[b] += V.Rti[0 + b] * gmu[0] + V.Rti[3 + b] * gmu[1] + V.Rti[6 + b] * gmu[2] - inv_m * g[kGvOcm + b];
        gs[am] += -ginvm * inv_m * inv_m;
        // G = Minv R_wc^T;  Minv[a][j] = R_q[j][a] / s_a
        for (int a = 0; a < 3; ++a)
            for (int j = 0; j < 3; ++j) {
                const double gM = gG[a][0] * Rw[0][j] + gG[a][1] * Rw[1][j] + gG[a][2] * Rw[2][j];
                gs[a] -= gM * Rq[j][a] / (s[a] * s[a]);
                gR[j][a] += gM / s[a];
            }
        for (int k = 0; k < 3; ++k) grgb[k] += g[kGvRgb + k];
    }
    // rotation matrix -> normalised quaternion
    double gw = 0, gx = 0, gy = 0, gz = 0;
    gx += -4 * x * (gR[1][1] + gR[2][2]);
    gy += -4 * y * (gR[0][0] + gR[2][2]);
    gz += -4 * z * (gR[0][0] + gR[1][1]);
    gx += 2 * y * gR[0][1]; gy += 2 * x * gR[0][1]; gw -= 2 * z * gR[0][1]; gz -= 2 * w * gR[0][1];
    gx += 2 * z * gR[0][2]; gz += 2 * x * gR[0][2]; gw += 2 * y * gR[0][2]; gy += 2 * w * gR[0][2];
    gx += 2 * y * gR[1][0]; gy += 2 * x * gR[1][0]; gw += 2 * z * gR[1][0]; gz += 2 * w * gR[1][0];
    gy += 2 * z * gR[1][2]; gz += 2 * y * gR[1][2]; gw -= 2 * x * gR[1][2]; gx -= 2 * w * gR[1][2];
    gx += 2 * z * gR[2][0]; gz += 2 * x * gR[2][0]; gw -= 2 * y * gR[2][0]; gy -= 2 * w * gR[2][0];
    gy += 2 * z * gR[2][1]; gz += 2 * y * gR[2][1]; gw += 2 * x * gR[2][1]; gx += 2 * w * gR[2][1];
    const double dot = gw * w + gx * x + gy * y + gz * z;
    float *O = g_geom + i * 16;
    O[0] += (float)gc[0];
    O[1] += (float)gc[1];
    O[2] += (float)gc[2];
    for (int a = 0; a < 3; ++a) O[3 + a] += (float)(gs[a] * s[a]);
    O[6] += (float)((gw - w * dot) * iq);
    O[7] += (float)((gx - x * dot) * iq);
    O[8] += (float)((gy - y * dot) * iq);
    O[9] += (float)((gz - z * dot) * iq);
    if (rgb_grad) {
        O[10] += (float)grgb[0];
        O[11] += (float)grgb[1];
        O[12] += (float)grgb[2];
    }
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_color_post(const void *__restrict__ net, int64_t n, int n_c, int off_feat,
                                                    int off_Wc1, int off_bc1, int stride,
                                                    const float *__restrict__ g_h0, float *__restrict__ g_net)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t base = i * stride;
    float f[kFeat], gf[kFeat];
#pragma unroll
    for (int k = 0; k < kFeat; ++k) {
        f[k] = ld_w<BF16>(net, base + off_feat + k);
        gf[k] = 0.0f;
    }
    for (int j = 0; j < n_c; ++j) {
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
    for (int k = 0; k < kFeat; ++k) g_net[base + off_feat + k] += gf[k];
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
    const unsigned g = (unsigned)((n + 255) / 256);
    if (bf16)
        k_color_post<true><<<g, 256, 0, st>>>(net, n, n_c, off_feat, off_Wc1, off_bc1, stride, g_h0, g_net);
    else
        k_color_post<false><<<g, 256, 0, st>>>(net, n, n_c, off_feat, off_Wc1, off_bc1, stride, g_h0, g_net);
    note_launch();
}

}  // namespace snp
