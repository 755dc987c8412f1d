// snp_grad.cu -- per-primitive gradient post-passes of the backward.
//
// k_project_bwd: the raster backward leaves, per (view, primitive), gradients of
// the projection record's geometry (Minv = diag(1/s) R(q)^T, op = Minv (eye - c),
// ocm = (eye - c)/m, 1/m with m = max(s)) and of the constant colour; this pass
// chains them to the centre, log-scales and quaternion (through its
// normalisation) and sums over views.
// k_color_post: the colour MLP's first layer is evaluated with the folded bias
// h0 = bc1 + Wc1[:, 3:] feat; this pass distributes dL/dh0 to bc1, Wc1[:, 3:]
// and feat.
#include "snp_common.cuh"
#include "snp_internal.h"

namespace snp {

constexpr int kGv = kGvFloats;

__global__ void __launch_bounds__(256) k_project_bwd(const float *__restrict__ geom, int64_t n,
                                                     const View *__restrict__ views, int n_views,
                                                     const float *__restrict__ g_view, float *__restrict__ g_geom)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *G = geom + i * 16;
    const float c[3] = {G[0], G[1], G[2]};
    const float ls[3] = {G[3], G[4], G[5]};
    const float q[4] = {G[6], G[7], G[8], G[9]};
    const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float iq = 1.0f / qn;
    const float w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (y * y + z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * (x * x + z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * (x * x + y * y);
    int am = 0;
    if (s[1] > s[am]) am = 1;
    if (s[2] > s[am]) am = 2;
    const float m = s[am], inv_m = 1.0f / m;
    const float is[3] = {1.0f / s[0], 1.0f / s[1], 1.0f / s[2]};

    float gc[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gR[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, grgb[3] = {0, 0, 0};
    for (int v = 0; v < n_views; ++v) {
        const float *g = g_view + ((int64_t)v * n + i) * kGv;
        const View &V = views[v];
        const float oc[3] = {V.eye[0] - c[0], V.eye[1] - c[1], V.eye[2] - c[2]};
        float gM[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) gM[a][b] = g[3 * a + b] + g[9 + a] * oc[b];
        float goc[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float t = g[12 + b] * inv_m;
#pragma unroll
            for (int a = 0; a < 3; ++a) t += R[b][a] * is[a] * g[9 + a];
            goc[b] = t;
        }
        const float ginvm = g[15] + g[12] * oc[0] + g[13] * oc[1] + g[14] * oc[2];
#pragma unroll
        for (int b = 0; b < 3; ++b) gc[b] -= goc[b];
        gs[am] += -ginvm * inv_m * inv_m;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                // Minv[a][b] = R[b][a] / s_a
                gs[a] -= gM[a][b] * R[b][a] * is[a] * is[a];
                gR[b][a] += gM[a][b] * is[a];
            }
#pragma unroll
        for (int k = 0; k < 3; ++k) grgb[k] += g[16 + k];
    }
    // rotation matrix -> normalised quaternion
    float gw = 0, gx = 0, gy = 0, gz = 0;
    gx += -4 * x * (gR[1][1] + gR[2][2]);
    gy += -4 * y * (gR[0][0] + gR[2][2]);
    gz += -4 * z * (gR[0][0] + gR[1][1]);
    // R01 = 2(xy - wz)
    gx += 2 * y * gR[0][1]; gy += 2 * x * gR[0][1]; gw -= 2 * z * gR[0][1]; gz -= 2 * w * gR[0][1];
    // R02 = 2(xz + wy)
    gx += 2 * z * gR[0][2]; gz += 2 * x * gR[0][2]; gw += 2 * y * gR[0][2]; gy += 2 * w * gR[0][2];
    // R10 = 2(xy + wz)
    gx += 2 * y * gR[1][0]; gy += 2 * x * gR[1][0]; gw += 2 * z * gR[1][0]; gz += 2 * w * gR[1][0];
    // R12 = 2(yz - wx)
    gy += 2 * z * gR[1][2]; gz += 2 * y * gR[1][2]; gw -= 2 * x * gR[1][2]; gx -= 2 * w * gR[1][2];
    // R20 = 2(xz - wy)
    gx += 2 * z * gR[2][0]; gz += 2 * x * gR[2][0]; gw -= 2 * y * gR[2][0]; gy -= 2 * w * gR[2][0];
    // R21 = 2(yz + wx)
    gy += 2 * z * gR[2][1]; gz += 2 * y * gR[2][1]; gw += 2 * x * gR[2][1]; gx += 2 * w * gR[2][1];
    const float dot = gw * w + gx * x + gy * y + gz * z;
    float *O = g_geom + i * 16;
    O[0] += gc[0];
    O[1] += gc[1];
    O[2] += gc[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) O[3 + a] += gs[a] * s[a];
    O[6] += (gw - w * dot) * iq;
    O[7] += (gx - x * dot) * iq;
    O[8] += (gy - y * dot) * iq;
    O[9] += (gz - z * dot) * iq;
    O[10] += grgb[0];
    O[11] += grgb[1];
    O[12] += grgb[2];
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
                        float *g_geom, cudaStream_t st)
{
    if (n <= 0) return;
    k_project_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(geom, n, views, n_views, g_view, g_geom);
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
