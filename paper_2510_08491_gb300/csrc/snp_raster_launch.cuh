// snp_raster_launch.cuh -- persistent launches of the raster kernels: the grid is
// the number of CTAs that fit on the device at once, and every CTA pulls tiles
// from the queue until it is exhausted.
#pragma once

#include <mutex>
#include <set>
#include <utility>

#include "snp_raster_bwd.cuh"
#include "snp_raster_fwd.cuh"

namespace snp {

constexpr size_t kSmemMax = 220 * 1024;

// Raise the dynamic shared-memory limit of a kernel once per (kernel, device)
// (before any stream capture: each kernel's first launch on a device is eager).
template <typename K>
static void allow_smem(K kern)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    const std::pair<const void *, int> key((const void *)kern, dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(key)) return;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    done.insert(key);
}

template <typename K>
static int persistent_grid(K kern, int threads, size_t smem, int64_t n_tiles, int tmem_per_sm = 0)
{
    int dev = 0, sms = 1, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (tmem_per_sm > 0) {
        // The occupancy query answers one CTA per SM for any kernel that allocates
        // tensor memory, whatever its registers and shared memory; the CTAs of this
        // one allocate a fixed share of the SM's columns (tmem_per_sm CTAs fit), so
        // count the resident CTAs from registers, shared memory and threads instead.
        cudaFuncAttributes fa{};
        int regs_sm = 65536, smem_sm = 0, resv = 0, thr_sm = 2048, blk_sm = 32;
        cudaFuncGetAttributes(&fa, kern);
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
        const int warps = (threads + 31) / 32;
        const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in 256s
        const size_t smem_blk = smem + fa.sharedSizeBytes + (size_t)resv;
        nb = tmem_per_sm;
        if (regs_warp > 0 && regs_sm / (warps * regs_warp) < nb) nb = regs_sm / (warps * regs_warp);
        if (smem_blk > 0 && (int)((size_t)smem_sm / smem_blk) < nb) nb = (int)((size_t)smem_sm / smem_blk);
        if (thr_sm / threads < nb) nb = thr_sm / threads;
        if (blk_sm < nb) nb = blk_sm;
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
    }
    note_raster_ctas(nb > 0 ? nb : 1);
    int64_t g = (int64_t)(nb > 0 ? nb : 1) * sms;
    if (g > n_tiles) g = n_tiles;
    return (int)(g > 0 ? g : 1);
}

template <int TS, int NC, int FORM, bool BF16>
static snp_status run_fwd(const RasterArgs &a, cudaStream_t st)
{
    const size_t smem = fwd_smem_bytes<TS>(NC, a.n_sigma, a.chunk);
    if (smem > kSmemMax || a.chunk < 1 || a.chunk > 64 || a.chunk > kMaxChunk / 2) return SNP_ERR_INVALID_ARG;
    if (a.n_tiles <= 0) return SNP_OK;
    auto kern = k_raster_fwd<TS, NC, FORM, BF16>;
    allow_smem(kern);
    const int grid = persistent_grid(kern, TileCfg<TS>::NT, smem, a.n_tiles);
    kern<<<grid, TileCfg<TS>::NT, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

template <int TS, int NC, int FORM, bool BF16, int NS = 0>
static snp_status run_bwd(const RasterArgs &a, cudaStream_t st)
{
    const size_t smem = bwd_smem_bytes<TS>(NC, a.n_sigma, a.chunk, a.stride);
    // (with the tensor-memory accumulators a chunk's entries land in the warps'
    // operand tiles at its end: at most tmem_max_chunk of them)
    if (smem > kSmemMax || a.chunk < 1 || a.chunk > 32 || a.chunk * (TS * TS / 32) > kMaskWords / 2 ||
        (bwd_tmem(TS, NC) && a.chunk > tmem_max_chunk(TileCfg<TS>::NT, NC)) || (NS > 0 && a.n_sigma != NS) ||
        a.stride != net_stride(a.n_sigma, NC, a.off_sh >= 0, a.off_wt >= 0))
        return SNP_ERR_INVALID_ARG;
    if (a.n_tiles <= 0) return SNP_OK;
    auto kern = k_raster_bwd<TS, NC, FORM, BF16, NS>;
    allow_smem(kern);
    // A CTA of the tensor-memory path allocates N_c x chunk columns (rounded up to a
    // power of two, at least 32) of the SM's 512: no more CTAs per SM than fit.
    int tm_per_sm = 0;
    if (bwd_tmem(TS, NC)) {
        int cols = 32;
        while (cols < NC * a.chunk) cols <<= 1;
        tm_per_sm = 512 / cols;
    }
    const int grid = persistent_grid(kern, TileCfg<TS>::NT, smem, a.n_tiles, tm_per_sm);
    kern<<<grid, TileCfg<TS>::NT, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

// Forms built for a tile size: the stable integral always, Eq. 8 literally when NAIVE.
template <int TS, bool NAIVE>
static snp_status dispatch_fwd(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    if (form == SNP_FORM_NAIVE && !NAIVE) return SNP_ERR_UNSUPPORTED;
#define SNP_FWD_CASE(NCV)                                                                          \
    if (nc == NCV) {                                                                               \
        if (form == SNP_FORM_STABLE)                                                               \
            return bf16 ? run_fwd<TS, NCV, 0, true>(a, st) : run_fwd<TS, NCV, 0, false>(a, st);    \
        if constexpr (NAIVE)                                                                       \
            return bf16 ? run_fwd<TS, NCV, 1, true>(a, st) : run_fwd<TS, NCV, 1, false>(a, st);    \
    }
    SNP_FWD_CASE(0)
    SNP_FWD_CASE(32)
    SNP_FWD_CASE(64)
#undef SNP_FWD_CASE
    return SNP_ERR_UNSUPPORTED;
}

template <int TS, bool NAIVE>
static snp_status dispatch_bwd(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st)
{
    if (form == SNP_FORM_NAIVE && !NAIVE) return SNP_ERR_UNSUPPORTED;
    // 16-pixel tiles, stable form, no colour network, n_sigma = 8 (the paper's
    // primitive): a kernel built for that n_sigma, whose 63 gradient values per pair
    // take two warp reduce-scatters instead of three (measured 42.5 -> 37.1 ms on
    // the speed-protocol backward).  Built for n_sigma = 16 with N_c = 32 and 32 with
    // N_c = 64 the same packing saves no or one reduce-scatter of four or seven, and
    // the fully unrolled loop measured 6% and 5% slower, so those keep the general
    // kernel.
    constexpr bool kSpec = TS == 16;
#define SNP_BWD_CASE(NCV, NSV)                                                                     \
    if (nc == NCV) {                                                                               \
        if constexpr (kSpec && NSV > 0) {                                                          \
            if (form == SNP_FORM_STABLE && a.n_sigma == NSV)                                       \
                return bf16 ? run_bwd<TS, NCV, 0, true, NSV>(a, st) : run_bwd<TS, NCV, 0, false, NSV>(a, st); \
        }                                                                                          \
        if (form == SNP_FORM_STABLE)                                                               \
            return bf16 ? run_bwd<TS, NCV, 0, true>(a, st) : run_bwd<TS, NCV, 0, false>(a, st);    \
        if constexpr (NAIVE)                                                                       \
            return bf16 ? run_bwd<TS, NCV, 1, true>(a, st) : run_bwd<TS, NCV, 1, false>(a, st);    \
    }
    SNP_BWD_CASE(0, 8)
    SNP_BWD_CASE(32, 0)
    SNP_BWD_CASE(64, 0)
#undef SNP_BWD_CASE
    return SNP_ERR_UNSUPPORTED;
}

}  // namespace snp
