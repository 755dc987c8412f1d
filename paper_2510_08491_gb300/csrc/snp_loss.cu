// snp_loss.cu -- mean squared image error and its gradient, the photometric loss
// of the differentiation workload (render vs. a target image).
//
// One pass: every block grid-strides over the values, writes
// dL/dimage_i = 2 (image_i - target_i) / n and leaves its partial sum of squares
// (FP64) in a context-owned slot; the block that finishes last sums the slots in
// a fixed order, so the loss is deterministic, and re-arms the completion counter
// for the next call.  No host synchronisation, no allocation: the call can be
// captured in a CUDA graph.
#include "snp_common.cuh"
#include "snp_internal.h"

namespace snp {

namespace {

constexpr int kLossThreads = 256;

__global__ void __launch_bounds__(kLossThreads) k_mse_loss(const float *__restrict__ img,
                                                           const float *__restrict__ tgt, int64_t n,
                                                           float *__restrict__ dL, float *__restrict__ loss,
                                                           double *__restrict__ part, unsigned *counter)
{
    const float scale = 2.0f / (float)n;
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = n >> 2;
    const bool vec = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(tgt) |
                       reinterpret_cast<uintptr_t>(dL)) & 15u) == 0;
    int64_t tail = 0;
    if (vec) {
        const float4 *i4 = reinterpret_cast<const float4 *>(img);
        const float4 *t4 = reinterpret_cast<const float4 *>(tgt);
        float4 *d4 = reinterpret_cast<float4 *>(dL);
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
            const float4 a = i4[q], b = t4[q];
            const float4 e = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
            d4[q] = make_float4(scale * e.x, scale * e.y, scale * e.z, scale * e.w);
            acc = fmaf(e.x, e.x, acc);
            acc = fmaf(e.y, e.y, acc);
            acc = fmaf(e.z, e.z, acc);
            acc = fmaf(e.w, e.w, acc);
        }
        tail = n4 << 2;
    }
    for (int64_t q = tail + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        const float e = img[q] - tgt[q];
        dL[q] = scale * e;
        acc = fmaf(e, e, acc);
    }
    // block sum in FP64, fixed order
    __shared__ double s_w[kLossThreads / 32];
    __shared__ bool s_last;
    double v = (double)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kLossThreads / 32; ++w) b += s_w[w];
        part[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double tot = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) tot += ((volatile double *)part)[b];
        *loss = (float)(tot / (double)n);
        *counter = 0u;
    }
}

}  // namespace

snp_status launch_mse_loss(const float *img, const float *tgt, int64_t n, float *dL, float *loss, double *part,
                           unsigned *counter, int max_blocks, cudaStream_t st)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SNP_ERR_CUDA;
    const int64_t want = (n / 4 + kLossThreads - 1) / kLossThreads;
    int blocks = (int)std::min<int64_t>(std::max<int64_t>(want, 1), std::min(4 * sms, max_blocks));
    k_mse_loss<<<blocks, kLossThreads, 0, st>>>(img, tgt, n, dL, loss, part, counter);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

}  // namespace snp
