// snp_internal.h -- host-side declarations shared by the libsnp translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "snp.h"

namespace snp {

// Kernels launched by this library in this process (snp_kernel_launches).
extern std::atomic<long long> g_launches;
inline void note_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

struct View;
struct NetLayout;

// snp_prep.cu
void launch_project(const float *geom, int64_t n, const View *views, int n_views, int ts, float *rec, int4 *trect,
                    uint32_t *counts, cudaStream_t st);
int64_t scan_temp_words(int64_t n);
void scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total, uint32_t *tmp, cudaStream_t st);
void launch_emit(const int4 *trect, const uint32_t *counts, const uint32_t *offsets, const float *rec, int64_t n,
                 const View *views, int n_views, uint64_t *keys, uint32_t *vals, int64_t cap, int32_t *flags,
                 cudaStream_t st);
int64_t sort_hist_words(int64_t n_bound);
bool radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, const uint32_t *d_n,
                int64_t n_bound, int nbits, uint32_t *hist, uint32_t *hist_scan, uint32_t *scan_tmp,
                cudaStream_t st);
void launch_clamp_count(const uint32_t *total, int64_t cap, uint32_t *out, cudaStream_t st);
void launch_tile_ranges(const uint64_t *keys, const uint32_t *d_n, int64_t n_bound, uint2 *ranges, cudaStream_t st);

// Arguments of the per-tile rasterizer (forward and backward).
struct RasterArgs {
    const float *rec;         // [V*n][kRecFloats]
    const uint32_t *vals;     // sorted values (view * n + primitive)
    const uint2 *ranges;      // [n_tiles]
    const void *net;          // [n][stride] weights
    const View *views;
    int32_t n_views;
    int32_t n_sigma;
    int64_t n;
    int64_t n_tiles;
    const int32_t *lay;       // unused on device (layout passed by value below)
    int32_t off_W1, off_b1, off_w2, off_b2, off_feat, off_Wc1, off_bc1, off_Wc2, off_bc2, off_Wc3, off_bc3, off_sh;
    int32_t off_wt;           // time-conditioned density: W_t [n_sigma] (-1: static scene)
    int32_t stride;
    float omega0;
    float t_min;
    float bg[3];
    int32_t chunk;
    // forward outputs / saved state
    float *image;             // concatenated HWC views
    float4 *px_state;         // [P]: composited colour (no background) xyz, optical depth w
    uint32_t *px_nwalk;       // [P]: list entries walked up to the last composited one
    unsigned long long *stats;  // [3]: candidates, hits, composited
    // backward inputs / outputs
    const float *dL_dimage;   // concatenated HWC views
    float *g_net;             // [n][stride] float32
    float *g_view;            // [V*n][16] per (view, primitive) geometry intermediates
    float *g_h0;              // [n][n_c] gradient of the folded first-layer bias
    // persistent scheduling
    int *work_counter;        // next queue item (zeroed before each launch)
    const uint32_t *queue;    // tile ids ordered by decreasing list length (NULL: 0..n_tiles-1)
    // composited pixels of every (tile, list entry) pair, one bit per pixel slot of the
    // tile: [K][tile pixels / 32] words indexed by the sorted key position (written by
    // the forward, read by the backward)
    uint32_t *cmask;
    // per-primitive network blocks in the staged shared-memory layout (k_pack_net)
    float *npack;             // [n][npack_stride]
    int32_t npack_stride;     // floats per primitive
    // colour store (colour-MLP scenes): the forward writes (colour, alpha_hat) of every
    // composited pair, per key in the order of its composited-mask bits, so that the
    // backward reads them instead of evaluating the colour network again.  NULL: off.
    float4 *colstore;         // [col_cap]
    uint32_t *key_off;        // [K] first colstore index of each key's pairs (kNoStore: not stored)
    unsigned long long *col_count;  // bump allocator of the forward (zeroed before it)
    uint32_t col_cap;         // capacity in pairs
    // alpha_hat store (scenes without a colour network): the same scheme with one
    // float per composited pair, in the colour store's buffer.  NULL: off.
    float *ahstore;
    // set to 1 by a kernel whose bounded device wait gave up (zeroed with each forward)
    int *wait_status;
    // test hook: the tensor-memory backward first waits, with a short limit, on a
    // barrier phase that nothing completes, so that a test can see the status
    int32_t test_stuck_wait;
};

constexpr uint32_t kNoStore = 0xffffffffu;
// Pairs a forward CTA takes from the colour store at a time (it hands out slices of
// the block to its chunks, so that the global allocator is touched once per block).
constexpr uint32_t kColBlock = 8192;

// snp_raster_*.cu
// CTAs per SM of the calling thread's last persistent raster launch (recorded when
// its grid is sized).
void note_raster_ctas(int per_sm);
int last_raster_ctas();
snp_status launch_raster_fwd(const RasterArgs &a, int color_mode, int n_c, int form, int bf16, int ts,
                             cudaStream_t st);
// snp_sh.cu
// off_sht: the degree-0 time series [12][3] of a time-conditioned scene (-1: none)
void launch_sh_color(const float *geom, const void *net, int bf16, int64_t n, const View *views, int n_views,
                     int off_sh, int off_sht, int stride, float *rec, cudaStream_t st);
void launch_sh_bwd(const float *geom, const void *net, int bf16, int64_t n, const View *views, int n_views,
                   int off_sh, int off_sht, int stride, const float *rec, const float *g_view, float *g_net,
                   float *g_geom, cudaStream_t st);

// snp_train.cu
struct PopFields {       // density-network fields of the gradient record
    int32_t off[5], size[5];
    int32_t count, stride;
};
struct PopThresholds {   // float32 forms of the population-control thresholds
    float grad, prune, log_grow, log_prune;
};
struct AdamConsts {
    float beta1, beta2, one_m_beta1, one_m_beta2, corr1, corr2, eps;
};
struct AdamNetFields {   // [off, end) and rate per snp_net_layout field (off < 0: absent)
    int32_t off[14], end[14];
    float lr[14];
    int32_t stride;
};
snp_status launch_popctl_stat(const float *g_net, int64_t n, const PopFields &f, float *sum, int32_t *count,
                              cudaStream_t st);
snp_status launch_popctl_plan(const float *geom, int64_t n, const float *sum, const int32_t *count,
                              const PopThresholds &t, int32_t *action, uint32_t *outs, cudaStream_t st);
snp_status launch_popctl_apply(const float *geom, const void *net, int64_t n, int row_bytes, const int32_t *action,
                               const uint32_t *off, const float *noise, float log_shrink, float *geom_out,
                               void *net_out, cudaStream_t st);
snp_status launch_geom_reg(const float *geom, int64_t n, float scale, float *g_geom, float *loss, double *part,
                           unsigned *counter, int max_blocks, cudaStream_t st);
snp_status launch_adam_geom(float *p, const float *g, float *m, float *v, int64_t n, const float lr[4],
                            const AdamConsts &c, cudaStream_t st);
snp_status launch_adam_net(float *p, void *pb, const float *g, float *m, float *v, int64_t n,
                           const AdamNetFields &f, const AdamConsts &c, cudaStream_t st);

// snp_loss.cu
constexpr int kLossSlots = 1024;
snp_status launch_mse_loss(const float *img, const float *tgt, int64_t n, float *dL, float *loss, double *part,
                           unsigned *counter, int max_blocks, cudaStream_t st);
snp_status launch_raster_bwd(const RasterArgs &a, int color_mode, int n_c, int form, int bf16, int ts,
                             cudaStream_t st);
size_t raster_fwd_smem(int color_mode, int n_c, int n_sigma, int chunk, int ts);
int raster_npack_stride(int color_mode, int n_c, int n_sigma);
snp_status launch_pack_net(const RasterArgs &a, int color_mode, int n_c, int bf16, cudaStream_t st);
size_t raster_bwd_smem(int color_mode, int n_c, int n_sigma, int chunk, int ts, bool dyn);
int raster_default_chunk(int color_mode, int n_c, int n_sigma, bool backward, int ts, bool dyn);
snp_status launch_fwd_ts8(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st);
snp_status launch_fwd_ts16(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st);
snp_status launch_fwd_ts32(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st);
snp_status launch_bwd_ts8(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st);
snp_status launch_bwd_ts16(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st);
snp_status launch_bwd_ts32(const RasterArgs &a, int nc, int form, int bf16, cudaStream_t st);
void launch_tile_queue(const uint2 *ranges, int64_t n_tiles, uint64_t *qkeys, uint32_t *qvals, uint32_t *d_n,
                       cudaStream_t st);

// snp_grad.cu
void launch_project_bwd(const float *geom, int64_t n, const View *views, int n_views, const float *g_view,
                        int rgb_grad, float *g_geom, cudaStream_t st);
void launch_color_post(const void *net, int bf16, int64_t n, int n_c, int off_feat, int off_Wc1, int off_bc1,
                       int stride, const float *g_h0, float *g_net, cudaStream_t st);

}  // namespace snp
