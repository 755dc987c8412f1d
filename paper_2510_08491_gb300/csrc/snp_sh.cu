// snp_sh.cu -- spherical-harmonic colour (Sec. 3.1: view-dependent colour in four
// bands of real spherical harmonics, 48 coefficients per primitive).
//
// k_sh_color (forward): per (view, primitive), the colour along the unit
// direction v from the camera centre to the primitive centre,
//   c = max(0, 1/2 + sum_{i<16} Y_i(v) sh[i]) per channel,
// written into the projection record, where the rasterizer reads constant
// colours.  k_sh_bwd (backward): per primitive, the raster's dL/dc of every view
// is chained to the coefficients (dL/dsh[i] = sum_views [c > 0] dL/dc Y_i(v)) and,
// through v = (c_prim - eye) / |c_prim - eye|, to the centre.
//
// Y_i are the real harmonics of degree l = 0..3 in tesseral form, index l^2 + l + m.
//
// Time-conditioned scenes (App. Applications, volumetric dynamic scenes): the
// degree-0 coefficient of each channel is sh[0] + sum_{j=1..4} a_j xi^j
// + sum_{j=1..4} (b_j cos(j xi) + c_j sin(j xi)), xi the view's timestamp; the
// 12 series coefficients per channel are stored [12][3] as a_1..4, b_1..4, c_1..4.
#include "snp_common.cuh"
#include "snp_internal.h"

namespace snp {

namespace {

// Normalisation constants: 1/2 sqrt(1/pi); sqrt(3/(4 pi)); 1/2 sqrt(15/pi);
// 1/4 sqrt(5/pi); 1/4 sqrt(15/pi); 1/4 sqrt(35/(2 pi)); 1/2 sqrt(105/pi);
// 1/4 sqrt(21/(2 pi)); 1/4 sqrt(7/pi); 1/4 sqrt(105/pi).
constexpr float kY0 = 0.28209479177387814f, kY1 = 0.4886025119029199f, kY2a = 1.0925484305920792f,
                kY2b = 0.31539156525252005f, kY2c = 0.5462742152960396f, kY3a = 0.5900435899266435f,
                kY3b = 2.890611442640554f, kY3c = 0.4570457994644658f, kY3d = 0.3731763325901154f,
                kY3e = 1.445305721320277f;

__device__ __forceinline__ void sh_eval(float x, float y, float z, float (&Y)[16])
{
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    Y[0] = kY0;
    Y[1] = kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = kY1 * x;
    Y[4] = kY2a * x * y;
    Y[5] = kY2a * y * z;
    Y[6] = kY2b * (3.0f * z2 - 1.0f);
    Y[7] = kY2a * x * z;
    Y[8] = kY2c * (x2 - y2);
    Y[9] = kY3a * y * (3.0f * x2 - y2);
    Y[10] = kY3b * x * y * z;
    Y[11] = kY3c * y * (5.0f * z2 - 1.0f);
    Y[12] = kY3d * z * (5.0f * z2 - 3.0f);
    Y[13] = kY3c * x * (5.0f * z2 - 1.0f);
    Y[14] = kY3e * z * (x2 - y2);
    Y[15] = kY3a * x * (x2 - 3.0f * y2);
}

// The 12 basis values of the degree-0 time series at xi: xi^j, cos(j xi), sin(j xi), j = 1..4.
__device__ __forceinline__ void time_basis(float xi, float (&B)[12])
{
    float p = xi;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        B[j] = p;
        p *= xi;
        sincosf((float)(j + 1) * xi, &B[8 + j], &B[4 + j]);
    }
}

// Gradient of sum_i g_i Y_i(x, y, z) with respect to (x, y, z) (the harmonics as
// polynomials in the components; the caller projects onto the tangent plane).
__device__ __forceinline__ float3 sh_grad(float x, float y, float z, const float (&g)[16])
{
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    gy += kY1 * g[1];
    gz += kY1 * g[2];
    gx += kY1 * g[3];
    gx += kY2a * y * g[4];
    gy += kY2a * x * g[4];
    gy += kY2a * z * g[5];
    gz += kY2a * y * g[5];
    gz += 6.0f * kY2b * z * g[6];
    gx += kY2a * z * g[7];
    gz += kY2a * x * g[7];
    gx += 2.0f * kY2c * x * g[8];
    gy -= 2.0f * kY2c * y * g[8];
    gx += 6.0f * kY3a * x * y * g[9];
    gy += 3.0f * kY3a * (x2 - y2) * g[9];
    gx += kY3b * y * z * g[10];
    gy += kY3b * x * z * g[10];
    gz += kY3b * x * y * g[10];
    gy += kY3c * (5.0f * z2 - 1.0f) * g[11];
    gz += 10.0f * kY3c * y * z * g[11];
    gz += kY3d * (15.0f * z2 - 3.0f) * g[12];
    gx += kY3c * (5.0f * z2 - 1.0f) * g[13];
    gz += 10.0f * kY3c * x * z * g[13];
    gx += 2.0f * kY3e * x * z * g[14];
    gy -= 2.0f * kY3e * y * z * g[14];
    gz += kY3e * (x2 - y2) * g[14];
    gx += 3.0f * kY3a * (x2 - y2) * g[15];
    gy -= 6.0f * kY3a * x * y * g[15];
    return make_float3(gx, gy, gz);
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_sh_color(const float *__restrict__ geom, const void *__restrict__ net,
                                                  int64_t n, const View *__restrict__ views, int n_views, int off_sh,
                                                  int off_sht, int stride, float *__restrict__ rec)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * n_views) return;
    const int64_t v = q / n, i = q - v * n;
    const View &V = views[v];
    const float *c = geom + i * SNP_GEOM_STRIDE;
    float dx = c[0] - V.eye[0], dy = c[1] - V.eye[1], dz = c[2] - V.eye[2];
    const float ir = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= ir;
    dy *= ir;
    dz *= ir;
    float Y[16];
    sh_eval(dx, dy, dz, Y);
    const int64_t base = i * stride + off_sh;
    float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int b = 0; b < 16; ++b)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) col[ch] = fmaf(Y[b], ld_w<BF16>(net, base + 3 * b + ch), col[ch]);
    if (off_sht >= 0) {
        float B[12];
        time_basis(V.time, B);
        const int64_t tb = i * stride + off_sht;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float dc = 0.0f;
#pragma unroll
            for (int j = 0; j < 12; ++j) dc = fmaf(B[j], ld_w<BF16>(net, tb + 3 * j + ch), dc);
            col[ch] = fmaf(Y[0], dc, col[ch]);
        }
    }
    float *r = rec + q * kRecFloats + kRecRgb;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) r[ch] = fmaxf(col[ch], 0.0f);
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_sh_bwd(const float *__restrict__ geom, const void *__restrict__ net,
                                                int64_t n, const View *__restrict__ views, int n_views, int off_sh,
                                                int off_sht, int stride, const float *__restrict__ rec,
                                                const float *__restrict__ g_view, float *__restrict__ g_net,
                                                float *__restrict__ g_geom)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *c = geom + i * SNP_GEOM_STRIDE;
    const int64_t base = i * stride + off_sh;
    float K[16][3], gK[16][3];
#pragma unroll
    for (int b = 0; b < 16; ++b)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            K[b][ch] = ld_w<BF16>(net, base + 3 * b + ch);
            gK[b][ch] = 0.0f;
        }
    float gT[12][3];
#pragma unroll
    for (int j = 0; j < 12; ++j)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gT[j][ch] = 0.0f;
    float3 gc = make_float3(0.f, 0.f, 0.f);
    for (int v = 0; v < n_views; ++v) {
        const int64_t q = (int64_t)v * n + i;
        const float *g = g_view + q * kGvFloats + kGvRgb;
        const float *col = rec + q * kRecFloats + kRecRgb;
        // dL/d(1/2 + sum Y sh) per channel: zero where the colour is clamped at 0
        float gch[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gch[ch] = col[ch] > 0.0f ? g[ch] : 0.0f;
        if (gch[0] == 0.0f && gch[1] == 0.0f && gch[2] == 0.0f) continue;
        const View &V = views[v];
        float dx = c[0] - V.eye[0], dy = c[1] - V.eye[1], dz = c[2] - V.eye[2];
        const float ir = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= ir;
        dy *= ir;
        dz *= ir;
        float Y[16], gY[16];
        sh_eval(dx, dy, dz, Y);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            gY[b] = 0.0f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                gK[b][ch] = fmaf(gch[ch], Y[b], gK[b][ch]);
                gY[b] = fmaf(gch[ch], K[b][ch], gY[b]);
            }
        }
        if (off_sht >= 0) {
            // the series enters as Y_0 dc: dL/d(series coefficient j) = dL/dc Y_0 B_j(xi)
            float B[12];
            time_basis(V.time, B);
#pragma unroll
            for (int j = 0; j < 12; ++j)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) gT[j][ch] = fmaf(gch[ch] * kY0, B[j], gT[j][ch]);
        }
        // v = w / |w|, w = c - eye:  dL/dw = (I - v v^T) dL/dv / |w|
        const float3 gv = sh_grad(dx, dy, dz, gY);
        const float vg = gv.x * dx + gv.y * dy + gv.z * dz;
        gc.x += (gv.x - vg * dx) * ir;
        gc.y += (gv.y - vg * dy) * ir;
        gc.z += (gv.z - vg * dz) * ir;
    }
    if (g_net) {
#pragma unroll
        for (int b = 0; b < 16; ++b)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) g_net[base + 3 * b + ch] += gK[b][ch];
        if (off_sht >= 0) {
            const int64_t tb = i * stride + off_sht;
#pragma unroll
            for (int j = 0; j < 12; ++j)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) g_net[tb + 3 * j + ch] += gT[j][ch];
        }
    }
    if (g_geom) {
        float *O = g_geom + i * SNP_GEOM_STRIDE;
        O[0] += gc.x;
        O[1] += gc.y;
        O[2] += gc.z;
    }
}

}  // namespace

void launch_sh_color(const float *geom, const void *net, int bf16, int64_t n, const View *views, int n_views,
                     int off_sh, int off_sht, int stride, float *rec, cudaStream_t st)
{
    const int64_t total = n * n_views;
    if (total <= 0) return;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (bf16) k_sh_color<true><<<blocks, 256, 0, st>>>(geom, net, n, views, n_views, off_sh, off_sht, stride, rec);
    else k_sh_color<false><<<blocks, 256, 0, st>>>(geom, net, n, views, n_views, off_sh, off_sht, stride, rec);
    note_launch();
}

void launch_sh_bwd(const float *geom, const void *net, int bf16, int64_t n, const View *views, int n_views,
                   int off_sh, int off_sht, int stride, const float *rec, const float *g_view, float *g_net,
                   float *g_geom, cudaStream_t st)
{
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (bf16)
        k_sh_bwd<true><<<blocks, 256, 0, st>>>(geom, net, n, views, n_views, off_sh, off_sht, stride, rec, g_view,
                                               g_net, g_geom);
    else
        k_sh_bwd<false><<<blocks, 256, 0, st>>>(geom, net, n, views, n_views, off_sh, off_sht, stride, rec, g_view,
                                                g_net, g_geom);
    note_launch();
}

}  // namespace snp
