// snp_train.cu -- the training-step services around the renderer: the
// population-control statistic, decision and scene rewrite (Sec. 3.3, Population
// Control), the anisotropy regulariser on the scale vectors (Sec. 3.3 Training,
// Sec. 5.3) and a fused Adam step over the geometry and network arrays.
//
// All of it is memory-bound streaming over per-primitive rows: one warp per
// primitive where a row is long (network records), one thread per element or per
// primitive elsewhere, 16-byte vector accesses on the network arrays.
#include <cuda_bf16.h>

#include "snp_common.cuh"
#include "snp_internal.h"

namespace snp {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------- statistic

// m_i = || gradient of the density network's fields ||_2 (W1, b1, w2, b2 and, for a
// time-conditioned scene, W_t); where m_i > 0: sum += m_i, count += 1.
__global__ void __launch_bounds__(kThreads) k_popctl_stat(const float *__restrict__ g, int64_t n, PopFields f,
                                                          float *__restrict__ sum, int32_t *__restrict__ count)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const float *row = g + i * f.stride;
    float acc = 0.0f;
    for (int k = 0; k < f.count; ++k)
        for (int j = lane; j < f.size[k]; j += 32) {
            const float v = row[f.off[k] + j];
            acc = fmaf(v, v, acc);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc > 0.0f) {
        sum[i] += sqrtf(acc);
        count[i] += 1;
    }
}

// ---------------------------------------------------------------- decision

__global__ void __launch_bounds__(kThreads) k_popctl_plan(const float *__restrict__ geom, int64_t n,
                                                          const float *__restrict__ sum,
                                                          const int32_t *__restrict__ count, PopThresholds t,
                                                          int32_t *__restrict__ action, uint32_t *__restrict__ outs)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *G = geom + i * SNP_GEOM_STRIDE;
    const float l = fmaxf(fmaxf(G[3], G[4]), G[5]);
    const int32_t c = count[i];
    const float s = sum[i];
    int a;
    if (l > t.log_prune) a = SNP_POP_PRUNE;
    else if (c > 0 && s >= __fmul_rn(t.grad, (float)c)) a = l <= t.log_grow ? SNP_POP_CLONE : SNP_POP_SPLIT;
    else if (c == 0 || s < __fmul_rn(t.prune, (float)c)) a = SNP_POP_PRUNE;
    else a = SNP_POP_KEEP;
    action[i] = a;
    outs[i] = a == SNP_POP_PRUNE ? 0u : (a == SNP_POP_KEEP ? 1u : 2u);
}

// ---------------------------------------------------------------- rewrite

// One warp per parent: lanes 0..15 write the geometry columns of its output rows,
// all lanes copy the network row as 16-byte pieces.
__global__ void __launch_bounds__(kThreads) k_popctl_apply(const float *__restrict__ geom,
                                                           const uint4 *__restrict__ net, int64_t n, int row16,
                                                           const int32_t *__restrict__ action,
                                                           const uint32_t *__restrict__ off,
                                                           const float *__restrict__ noise, float log_shrink,
                                                           float *__restrict__ geom_out, uint4 *__restrict__ net_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int a = action[i];
    if (a == SNP_POP_PRUNE) return;
    const int outs = a == SNP_POP_KEEP ? 1 : 2;
    const int64_t o0 = off[i];
    const float *G = geom + i * SNP_GEOM_STRIDE;
    for (int j = 0; j < outs; ++j) {
        const int64_t o = o0 + j;
        if (lane < SNP_GEOM_STRIDE) {
            float v = G[lane];
            if (a == SNP_POP_SPLIT) {
                if (lane < 3) {
                    // child centre c + R(q) diag(s) eps_j, row `lane` of R
                    float qw = G[6], qx = G[7], qy = G[8], qz = G[9];
                    const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
                    qw *= qn;
                    qx *= qn;
                    qy *= qn;
                    qz *= qn;
                    float r0, r1, r2;
                    if (lane == 0) {
                        r0 = 1.0f - 2.0f * (qy * qy + qz * qz);
                        r1 = 2.0f * (qx * qy - qw * qz);
                        r2 = 2.0f * (qx * qz + qw * qy);
                    } else if (lane == 1) {
                        r0 = 2.0f * (qx * qy + qw * qz);
                        r1 = 1.0f - 2.0f * (qx * qx + qz * qz);
                        r2 = 2.0f * (qy * qz - qw * qx);
                    } else {
                        r0 = 2.0f * (qx * qz - qw * qy);
                        r1 = 2.0f * (qy * qz + qw * qx);
                        r2 = 1.0f - 2.0f * (qx * qx + qy * qy);
                    }
                    const float *e = noise + (i * 2 + j) * 3;
                    v += r0 * expf(G[3]) * e[0] + r1 * expf(G[4]) * e[1] + r2 * expf(G[5]) * e[2];
                } else if (lane < 6) {
                    v = __fsub_rn(v, log_shrink);
                }
            }
            geom_out[o * SNP_GEOM_STRIDE + lane] = v;
        }
        const uint4 *src = net + i * row16;
        uint4 *dst = net_out + o * row16;
        for (int q = lane; q < row16; q += 32) dst[q] = src[q];
    }
}

// ---------------------------------------------------------------- regulariser

__global__ void __launch_bounds__(kThreads) k_geom_reg(const float *__restrict__ geom, int64_t n, float scale,
                                                       float *__restrict__ g_geom, float *__restrict__ loss,
                                                       double *__restrict__ part, unsigned *counter)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float *G = geom + i * SNP_GEOM_STRIDE;
        const float s0 = expf(G[3]), s1 = expf(G[4]), s2 = expf(G[5]);
        // s_a - mean(s) from the pairwise differences (exact for close scales, and
        // exactly 0 for an isotropic primitive, where std has no derivative)
        const float e01 = s0 - s1, e02 = s0 - s2, e12 = s1 - s2;
        const float d0 = (e01 + e02) * (1.0f / 3.0f), d1 = (e12 - e01) * (1.0f / 3.0f),
                    d2 = -(e02 + e12) * (1.0f / 3.0f);
        const float sd = sqrtf((d0 * d0 + d1 * d1 + d2 * d2) * (1.0f / 3.0f));
        acc += (double)sd;
        if (g_geom && sd > 0.0f) {
            // d std / d s_a = (s_a - mu) / (3 std); d s_a / d log s_a = s_a
            const float k = scale / (3.0f * sd);
            float *O = g_geom + i * SNP_GEOM_STRIDE + 3;
            O[0] += k * s0 * d0;
            O[1] += k * s1 * d1;
            O[2] += k * s2 * d2;
        }
    }
    __shared__ double s_w[kThreads / 32];
    __shared__ bool s_last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) b += s_w[w];
        part[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double tot = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) tot += ((volatile double *)part)[b];
        *loss = (float)(tot * (double)scale);
        *counter = 0u;
    }
}

// ---------------------------------------------------------------- Adam

__device__ __forceinline__ float adam_update(float p, float g, float &m, float &v, float lr, const AdamConsts &c)
{
    m = fmaf(c.beta1, m, c.one_m_beta1 * g);
    v = fmaf(c.beta2, v, c.one_m_beta2 * g * g);
    return p - lr * (m * c.corr1) / (sqrtf(v * c.corr2) + c.eps);
}

// Geometry [n][16]: one thread per element; the column picks the rate.
__global__ void __launch_bounds__(kThreads) k_adam_geom(float *__restrict__ p, const float *__restrict__ g,
                                                        float *__restrict__ m, float *__restrict__ v, int64_t total,
                                                        float4 lr, AdamConsts c)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(q & (SNP_GEOM_STRIDE - 1));
        if (col >= 13) continue;
        const float r = col < 3 ? lr.x : (col < 6 ? lr.y : (col < 10 ? lr.z : lr.w));
        float mm = m[q], vv = v[q];
        p[q] = adam_update(p[q], g[q], mm, vv, r, c);
        m[q] = mm;
        v[q] = vv;
    }
}

// Network [n][stride]: one thread per 4 consecutive elements (16-byte accesses).
// Fields start on multiples of 8 elements, so a group of 4 never straddles two
// fields; groups past the last field (tail padding) are skipped.
template <bool BF16>
__global__ void __launch_bounds__(kThreads) k_adam_net(float *__restrict__ p, __nv_bfloat16 *__restrict__ pb,
                                                       const float *__restrict__ g, float *__restrict__ m,
                                                       float *__restrict__ v, int64_t n, AdamNetFields f,
                                                       AdamConsts c)
{
    const int g4 = f.stride / 4;
    const int64_t total = n * g4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)(q % g4) * 4;
        float lr = -1.0f;
#pragma unroll
        for (int k = 0; k < 14; ++k)
            if (f.off[k] >= 0 && col >= f.off[k] && col < f.end[k]) lr = f.lr[k];
        if (lr < 0.0f) continue;
        float4 P = reinterpret_cast<const float4 *>(p)[q];
        const float4 Gv = reinterpret_cast<const float4 *>(g)[q];
        float4 M = reinterpret_cast<const float4 *>(m)[q];
        float4 V = reinterpret_cast<const float4 *>(v)[q];
        P.x = adam_update(P.x, Gv.x, M.x, V.x, lr, c);
        P.y = adam_update(P.y, Gv.y, M.y, V.y, lr, c);
        P.z = adam_update(P.z, Gv.z, M.z, V.z, lr, c);
        P.w = adam_update(P.w, Gv.w, M.w, V.w, lr, c);
        reinterpret_cast<float4 *>(p)[q] = P;
        reinterpret_cast<float4 *>(m)[q] = M;
        reinterpret_cast<float4 *>(v)[q] = V;
        if constexpr (BF16) {
            const __nv_bfloat162 lo = __floats2bfloat162_rn(P.x, P.y), hi = __floats2bfloat162_rn(P.z, P.w);
            uint2 w;
            w.x = *reinterpret_cast<const uint32_t *>(&lo);
            w.y = *reinterpret_cast<const uint32_t *>(&hi);
            reinterpret_cast<uint2 *>(pb)[q] = w;
        }
    }
}

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

unsigned stream_blocks(int64_t work)
{
    const int sms = sm_count();
    const int64_t want = (work + kThreads - 1) / kThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)8 * (sms > 0 ? sms : 152)));
}

}  // namespace

snp_status launch_popctl_stat(const float *g_net, int64_t n, const PopFields &f, float *sum, int32_t *count,
                              cudaStream_t st)
{
    if (n <= 0) return SNP_OK;
    k_popctl_stat<<<(unsigned)((n * 32 + kThreads - 1) / kThreads), kThreads, 0, st>>>(g_net, n, f, sum, count);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

snp_status launch_popctl_plan(const float *geom, int64_t n, const float *sum, const int32_t *count,
                              const PopThresholds &t, int32_t *action, uint32_t *outs, cudaStream_t st)
{
    if (n <= 0) return SNP_OK;
    k_popctl_plan<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(geom, n, sum, count, t, action,
                                                                                 outs);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

snp_status launch_popctl_apply(const float *geom, const void *net, int64_t n, int row_bytes, const int32_t *action,
                               const uint32_t *off, const float *noise, float log_shrink, float *geom_out,
                               void *net_out, cudaStream_t st)
{
    if (n <= 0) return SNP_OK;
    k_popctl_apply<<<(unsigned)((n * 32 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        geom, (const uint4 *)net, n, row_bytes / 16, action, off, noise, log_shrink, geom_out, (uint4 *)net_out);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

snp_status launch_geom_reg(const float *geom, int64_t n, float scale, float *g_geom, float *loss, double *part,
                           unsigned *counter, int max_blocks, cudaStream_t st)
{
    const unsigned blocks = std::min<unsigned>(stream_blocks(n), (unsigned)max_blocks);
    k_geom_reg<<<blocks, kThreads, 0, st>>>(geom, n, scale, g_geom, loss, part, counter);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

snp_status launch_adam_geom(float *p, const float *g, float *m, float *v, int64_t n, const float lr[4],
                            const AdamConsts &c, cudaStream_t st)
{
    if (n <= 0) return SNP_OK;
    const int64_t total = n * SNP_GEOM_STRIDE;
    k_adam_geom<<<stream_blocks(total), kThreads, 0, st>>>(p, g, m, v, total, make_float4(lr[0], lr[1], lr[2], lr[3]),
                                                           c);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

snp_status launch_adam_net(float *p, void *pb, const float *g, float *m, float *v, int64_t n,
                           const AdamNetFields &f, const AdamConsts &c, cudaStream_t st)
{
    if (n <= 0) return SNP_OK;
    const unsigned blocks = stream_blocks(n * (f.stride / 4));
    if (pb)
        k_adam_net<true><<<blocks, kThreads, 0, st>>>(p, (__nv_bfloat16 *)pb, g, m, v, n, f, c);
    else
        k_adam_net<false><<<blocks, kThreads, 0, st>>>(p, nullptr, g, m, v, n, f, c);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

}  // namespace snp
