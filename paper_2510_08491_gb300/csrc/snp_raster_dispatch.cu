// snp_raster_dispatch.cu -- tile-size dispatch of the raster kernels, their
// shared-memory sizing and default chunk, and the length-ordered tile queue.
#include "snp_raster_bwd.cuh"
#include "snp_raster_fwd.cuh"

namespace snp {

static int nc_of(int color_mode, int n_c) { return color_mode == SNP_COLOR_MLP ? n_c : 0; }

size_t raster_fwd_smem(int color_mode, int n_c, int n_sigma, int chunk, int ts)
{
    const int nc = nc_of(color_mode, n_c);
    if (ts == 8) return fwd_smem_bytes<8>(nc, n_sigma, chunk);
    if (ts == 32) return fwd_smem_bytes<32>(nc, n_sigma, chunk);
    return fwd_smem_bytes<16>(nc, n_sigma, chunk);
}

size_t raster_bwd_smem(int color_mode, int n_c, int n_sigma, int chunk, int ts, bool dyn)
{
    const int nc = nc_of(color_mode, n_c);
    const int stride = net_stride(n_sigma, nc, color_mode == SNP_COLOR_SH, dyn);
    if (ts == 8) return bwd_smem_bytes<8>(nc, n_sigma, chunk, stride);
    if (ts == 32) return bwd_smem_bytes<32>(nc, n_sigma, chunk, stride);
    return bwd_smem_bytes<16>(nc, n_sigma, chunk, stride);
}

// Largest chunk (<= 32 forward; backward <= 32 at 16-pixel tiles, else <= 8)
// within the shared-memory budget: for k CTAs per SM, k (dynamic + static + the
// 1 KB per-CTA reservation) must fit the SM's 228 KB, so the dynamic part of one
// CTA stays below 228 KB / k - 1 KB - its static shared memory (about 2.6 KB in the
// forward, 4.8 KB in the backward).  A budget above that silently drops a CTA per
// SM: the time-conditioned backward at chunk 15 (108.7 KB) ran one CTA per SM and
// took 55.6 ms against 36.8 ms at chunk 8.
int raster_default_chunk(int color_mode, int n_c, int n_sigma, bool backward, int ts, bool dyn)
{
    const int fmb = fwd_min_blocks(ts, nc_of(color_mode, n_c));
    // (at 16-pixel tiles and N_c = 32 the 72 KB budget gives chunk 5, 71.5 KB, which
    // fits three CTAs per SM and measured faster than chunk 4: 22.3 against 23.2 ms at
    // the four-view 1080p workload)
    const size_t fwd_budget = fmb == 4 ? 52 * 1024 : (fmb == 3 ? 72 * 1024 : 104 * 1024);
    // (the tensor-memory backward at N_c = 64 also holds its operand tiles: most of one SM)
    const size_t bwd_budget = bwd_min_blocks(ts, nc_of(color_mode, n_c)) == 2
                                  ? 108 * 1024
                                  : (bwd_tmem(ts, nc_of(color_mode, n_c)) ? 220 * 1024 : 200 * 1024);
    int ch = backward ? (ts == 16 ? 32 : 8) : 32;
    if (backward && bwd_tmem(ts, nc_of(color_mode, n_c)))
        ch = tmem_max_chunk(ts == 8 ? 64 : 256, nc_of(color_mode, n_c));
    if (backward) {
        while (ch > 1 && raster_bwd_smem(color_mode, n_c, n_sigma, ch, ts, dyn) > bwd_budget) --ch;
    } else {
        while (ch > 1 && raster_fwd_smem(color_mode, n_c, n_sigma, ch, ts) > fwd_budget) --ch;
    }
    return ch;
}

static thread_local int t_raster_ctas = 0;
void note_raster_ctas(int per_sm) { t_raster_ctas = per_sm; }
int last_raster_ctas() { return t_raster_ctas; }

int raster_npack_stride(int color_mode, int n_c, int n_sigma)
{
    return den_stride(n_sigma) + col_stride(nc_of(color_mode, n_c));
}

template <int NC, bool BF16>
static snp_status run_pack(const RasterArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return SNP_OK;
    const int64_t blocks = (a.n * 32 + 255) / 256;
    k_pack_net<NC, BF16><<<(unsigned)blocks, 256, 0, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

snp_status launch_pack_net(const RasterArgs &a, int color_mode, int n_c, int bf16, cudaStream_t st)
{
    const int nc = nc_of(color_mode, n_c);
    if (nc == 0) return bf16 ? run_pack<0, true>(a, st) : run_pack<0, false>(a, st);
    if (nc == 32) return bf16 ? run_pack<32, true>(a, st) : run_pack<32, false>(a, st);
    if (nc == 64) return bf16 ? run_pack<64, true>(a, st) : run_pack<64, false>(a, st);
    return SNP_ERR_UNSUPPORTED;
}

snp_status launch_raster_fwd(const RasterArgs &a, int color_mode, int n_c, int form, int bf16, int ts,
                             cudaStream_t st)
{
    const int nc = nc_of(color_mode, n_c);
    if (ts == 8) return launch_fwd_ts8(a, nc, form, bf16, st);
    if (ts == 16) return launch_fwd_ts16(a, nc, form, bf16, st);
    if (ts == 32) return launch_fwd_ts32(a, nc, form, bf16, st);
    return SNP_ERR_UNSUPPORTED;
}

snp_status launch_raster_bwd(const RasterArgs &a, int color_mode, int n_c, int form, int bf16, int ts,
                             cudaStream_t st)
{
    const int nc = nc_of(color_mode, n_c);
    if (ts == 8) return launch_bwd_ts8(a, nc, form, bf16, st);
    if (ts == 16) return launch_bwd_ts16(a, nc, form, bf16, st);
    if (ts == 32) return launch_bwd_ts32(a, nc, form, bf16, st);
    return SNP_ERR_UNSUPPORTED;
}

// Queue keys: (0xffffffff - list length) so that an ascending sort puts the
// longest tile lists first; value = tile id.
__global__ void __launch_bounds__(256) k_tile_queue_keys(const uint2 *__restrict__ ranges, int64_t n_tiles,
                                                         uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                         uint32_t *__restrict__ d_n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *d_n = (uint32_t)n_tiles;
    if (t >= n_tiles) return;
    const uint2 r = ranges[t];
    keys[t] = (uint64_t)(0xffffffffu - (r.y - r.x));
    vals[t] = (uint32_t)t;
}

void launch_tile_queue(const uint2 *ranges, int64_t n_tiles, uint64_t *qkeys, uint32_t *qvals, uint32_t *d_n,
                       cudaStream_t st)
{
    if (n_tiles <= 0) return;
    k_tile_queue_keys<<<(unsigned)((n_tiles + 255) / 256), 256, 0, st>>>(ranges, n_tiles, qkeys, qvals, d_n);
    note_launch();
}

}  // namespace snp
