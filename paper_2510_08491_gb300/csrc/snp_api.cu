// snp_api.cu -- the C ABI declared in include/snp.h: context, workspace,
// forward/backward orchestration on one stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "snp.h"
#include "snp_common.cuh"
#include "snp_internal.h"

using namespace snp;

std::atomic<long long> snp::g_launches{0};

namespace {

// CUDA events around stages; elapsed times are collected lazily.
struct StageTimer {
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Pending> pending;
    double ms[SNP_N_STAGES] = {};
    int64_t calls[SNP_N_STAGES] = {};
    cudaEvent_t open_ev = nullptr;
    int open_stage = -1;

    cudaEvent_t get()
    {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void begin(int stage, cudaStream_t st)
    {
        open_ev = get();
        open_stage = stage;
        cudaEventRecord(open_ev, st);
    }
    void end(cudaStream_t st)
    {
        if (open_stage < 0) return;
        cudaEvent_t b = get();
        cudaEventRecord(b, st);
        pending.push_back({open_stage, open_ev, b});
        open_stage = -1;
        if (pending.size() > 4096) collect();
    }
    void collect()
    {
        if (pending.empty()) return;
        cudaEventSynchronize(pending.back().b);
        for (auto &p : pending) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                ms[p.stage] += t;
                calls[p.stage] += 1;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    void destroy()
    {
        collect();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

int round8(int x) { return (x + 7) & ~7; }

void layout_of(const snp_scene_desc &d, snp_net_layout &L)
{
    int off = 0;
    const int ns = d.n_sigma;
    for (int k = 0; k < 14; ++k) L.off[k] = -1;
    L.off[0] = off; off += round8(3 * ns);
    L.off[1] = off; off += round8(ns);
    L.off[2] = off; off += round8(ns);
    L.off[3] = off; off += 8;
    if (d.color_mode == SNP_COLOR_MLP) {
        const int nc = d.n_c;
        L.off[4] = off; off += round8(kFeat);
        L.off[5] = off; off += round8(nc * (3 + kFeat));
        L.off[6] = off; off += round8(nc);
        L.off[7] = off; off += round8(nc * nc);
        L.off[8] = off; off += round8(nc);
        L.off[9] = off; off += round8(3 * nc);
        L.off[10] = off; off += 8;
    }
    if (d.color_mode == SNP_COLOR_SH) {
        L.off[11] = off; off += 48;
    }
    if (d.dynamic) {
        L.off[12] = off; off += round8(ns);
        if (d.color_mode == SNP_COLOR_SH) {
            L.off[13] = off; off += round8(36);
        }
    }
    L.stride = off;
}

int tile_bits(int64_t tiles)
{
    int b = 1;
    while (((int64_t)1 << b) < tiles) ++b;
    return b;
}

}  // namespace

struct snp_context {
    int device = 0;
    int fwd_ctas = 0, bwd_ctas = 0;  // CTAs per SM of the last raster launches
    std::mutex mu;
    char err[512] = {0};
    bool reserved = false;
    // device workspace
    Buf views, rec, trect, counts, offsets, scan_tmp, keys, vals, keys_alt, vals_alt, hist, hist_scan, ranges,
        px_state, px_nwalk, stats, small, g_view, g_h0, qkeys, qvals, qkeys_alt, qvals_alt, qhist, qhist_scan, npack,
        cmask;
    // loss reduction: kLossSlots FP64 block sums, then the completion counter
    Buf loss_part;
    // population-control plan: per-primitive output counts, scan scratch, total
    Buf pop_cnt, pop_tmp, pop_total;
    // colour store of the latest forward (colour-MLP scenes) and its per-key offsets
    Buf colstore, key_off;
    bool col_on = false;       // the latest forward wrote the store
    int64_t last_comp = 0;     // composited pairs of the previous forward (sizes the store)
    bool fwd_done = false;     // the stats buffer holds a finished forward's counters
    // pinned host staging
    View *h_views = nullptr;
    uint32_t *h_small = nullptr;
    cudaEvent_t ev_views = nullptr;
    // state of the latest forward
    int64_t token = 0;
    int64_t K = 0, key_cap = 0;
    bool keys_in_alt = false;
    int n_views = 0;
    int64_t n = 0, n_tiles = 0, n_pixels = 0;
    snp_scene_desc desc{};
    snp_config cfg{};
    int ts = 16, chunk = 0;
    bool queue_in_alt = false;
    StageTimer timer;
    bool timing = false;
    // cameras of the reservation (a captured forward must use exactly these)
    snp_camera res_cams[kMaxViews];
    int res_n_cams = 0, res_ts = 16;
    int64_t res_tiles = 0, res_pixels = 0;
};

// Offsets inside the small device buffer.
constexpr size_t kSmallTotal = 0, kSmallFlags = 16, kSmallTiles = 32, kSmallWork = 48, kSmallNsort = 64,
                 kSmallColCount = 128, kSmallBytes = 256;

// Host-side NVTX range per stage (visible to Nsight tools and to ncu's
// --nvtx-include filters), plus CUDA events when stage timing is on.
static const char *const kStageNames[SNP_N_STAGES] = {"snp:project", "snp:scan",       "snp:emit",
                                                      "snp:sort",    "snp:ranges",     "snp:raster_fwd",
                                                      "snp:raster_bwd", "snp:post_bwd"};
#define STAGE_BEGIN(k)                        \
    do {                                      \
        nvtxRangePushA(kStageNames[(k)]);     \
        if (ctx->timing) ctx->timer.begin((k), st); \
    } while (0)
#define STAGE_END()                           \
    do {                                      \
        if (ctx->timing) ctx->timer.end(st);  \
        nvtxRangePop();                       \
    } while (0)

static snp_status fail(snp_context *c, snp_status s, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return fail(ctx, SNP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static snp_status ensure(snp_context *ctx, Buf &b, size_t bytes, const char *name)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return SNP_OK;
    if (ctx->reserved)
        return fail(ctx, SNP_ERR_CAPACITY, "workspace '%s' needs %zu bytes, reserved %zu", name, bytes, b.bytes);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    const size_t want = bytes + bytes / 4;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) return fail(ctx, SNP_ERR_CUDA, "cudaMalloc(%s, %zu): %s", name, want, cudaGetErrorString(e));
    b.bytes = want;
    return SNP_OK;
}

#define ENS(buf, bytes)                                            \
    do {                                                           \
        snp_status s_ = ensure(ctx, ctx->buf, (bytes), #buf);      \
        if (s_ != SNP_OK) return s_;                               \
    } while (0)

static snp_status check_desc(snp_context *ctx, const snp_scene_desc *d)
{
    if (!d) return fail(ctx, SNP_ERR_INVALID_ARG, "desc is NULL");
    if (d->n < 0 || d->n > (int64_t)1 << 28) return fail(ctx, SNP_ERR_INVALID_ARG, "n out of range: %lld", (long long)d->n);
    if (d->n_sigma < 1 || d->n_sigma > 64) return fail(ctx, SNP_ERR_INVALID_ARG, "n_sigma out of range: %d", d->n_sigma);
    if (d->color_mode != SNP_COLOR_CONST && d->color_mode != SNP_COLOR_MLP && d->color_mode != SNP_COLOR_SH)
        return fail(ctx, SNP_ERR_INVALID_ARG, "bad color_mode %d", d->color_mode);
    if (d->color_mode == SNP_COLOR_MLP && d->n_c != 32 && d->n_c != 64)
        return fail(ctx, SNP_ERR_UNSUPPORTED, "n_c must be 32 or 64, got %d", d->n_c);
    if (d->weight_dtype != SNP_F32 && d->weight_dtype != SNP_BF16)
        return fail(ctx, SNP_ERR_INVALID_ARG, "bad weight_dtype %d", d->weight_dtype);
    if (d->dynamic != 0 && d->dynamic != 1) return fail(ctx, SNP_ERR_INVALID_ARG, "bad dynamic flag %d", d->dynamic);
    if (d->dynamic && d->color_mode == SNP_COLOR_MLP)
        return fail(ctx, SNP_ERR_UNSUPPORTED, "time-conditioned scenes are built for constant or SH colour");
    return SNP_OK;
}

static snp_status check_cams(snp_context *ctx, const snp_camera *cams, int n_cams)
{
    if (!cams || n_cams < 1 || n_cams > kMaxViews)
        return fail(ctx, SNP_ERR_INVALID_ARG, "need 1..%d cameras, got %d", kMaxViews, n_cams);
    for (int v = 0; v < n_cams; ++v) {
        const snp_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768)
            return fail(ctx, SNP_ERR_INVALID_ARG, "camera %d: bad size %dx%d", v, c.width, c.height);
        if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !(c.z_near > 0.0f))
            return fail(ctx, SNP_ERR_INVALID_ARG, "camera %d: fx, fy, z_near must be > 0", v);
        if (!std::isfinite(c.time)) return fail(ctx, SNP_ERR_INVALID_ARG, "camera %d: time is not finite", v);
    }
    return SNP_OK;
}

// A tile key's value is the (view, primitive) instance v * n + i and the key offsets
// are scanned in 32 bits, so both must fit in uint32.
static snp_status check_instances(snp_context *ctx, int64_t n, int n_cams)
{
    if (n * (int64_t)n_cams > (int64_t)0xffffffff)
        return fail(ctx, SNP_ERR_UNSUPPORTED, "n x views = %lld exceeds the 32-bit instance index",
                    (long long)(n * (int64_t)n_cams));
    return SNP_OK;
}

// Fill the pinned view table for these cameras; returns tiles and pixels.
static snp_status build_views(snp_context *ctx, const snp_camera *cams, int n_cams, int ts, int64_t *tiles,
                              int64_t *pixels)
{
    if (ctx->ev_views) CK(cudaEventSynchronize(ctx->ev_views));
    int64_t t = 0, p = 0;
    for (int v = 0; v < n_cams; ++v) {
        View &V = ctx->h_views[v];
        const snp_camera &c = cams[v];
        memcpy(V.R, c.R_wc, sizeof(V.R));
        memcpy(V.eye, c.eye, sizeof(V.eye));
        V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy; V.z_near = c.z_near;
        V.width = c.width; V.height = c.height;
        V.tiles_x = (c.width + ts - 1) / ts;
        V.tiles_y = (c.height + ts - 1) / ts;
        V.tile_off = (int32_t)t;
        V.time = c.time;
        V.pix_off = p;
        {
            // (R_wc^T)^-1 by the adjugate, in FP64
            double M[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) M[a][b] = (double)c.R_wc[3 * b + a];  // R_wc^T
            const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                               M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            if (!(fabs(det) > 1e-6)) return fail(ctx, SNP_ERR_INVALID_ARG, "camera %d: R_wc is singular", v);
            const double id = 1.0 / det;
            double I[3][3];
            I[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) * id;
            I[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) * id;
            I[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) * id;
            I[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) * id;
            I[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) * id;
            I[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) * id;
            I[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) * id;
            I[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) * id;
            I[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) * id;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    V.Rti[3 * a + b] = I[a][b];
                    V.Rti_hi[3 * a + b] = (float)I[a][b];
                    V.Rti_lo[3 * a + b] = (float)(I[a][b] - (double)V.Rti_hi[3 * a + b]);
                }
        }
        t += (int64_t)V.tiles_x * V.tiles_y;
        p += (int64_t)c.width * c.height;
    }
    if (t >= ((int64_t)1 << 31)) return fail(ctx, SNP_ERR_INVALID_ARG, "too many tiles");
    *tiles = t;
    *pixels = p;
    return SNP_OK;
}

static void fill_args(RasterArgs &a, const snp_context *ctx, const snp_scene_desc *d, const snp_scene_ptrs *sc,
                      const uint32_t *sorted_vals)
{
    memset(&a, 0, sizeof(a));
    snp_net_layout L;
    layout_of(*d, L);
    a.rec = (const float *)ctx->rec.p;
    a.vals = sorted_vals;
    a.ranges = (const uint2 *)ctx->ranges.p;
    a.net = sc->net;
    a.views = (const View *)ctx->views.p;
    a.n_views = ctx->n_views;
    a.n_sigma = d->n_sigma;
    a.n = d->n;
    a.n_tiles = ctx->n_tiles;
    a.off_W1 = L.off[0]; a.off_b1 = L.off[1]; a.off_w2 = L.off[2]; a.off_b2 = L.off[3];
    a.off_feat = L.off[4]; a.off_Wc1 = L.off[5]; a.off_bc1 = L.off[6]; a.off_Wc2 = L.off[7];
    a.off_bc2 = L.off[8]; a.off_Wc3 = L.off[9]; a.off_bc3 = L.off[10]; a.off_sh = L.off[11];
    a.off_wt = L.off[12];
    a.stride = L.stride;
    a.omega0 = d->omega0;
    a.t_min = ctx->cfg.t_min;
    for (int k = 0; k < 3; ++k) a.bg[k] = ctx->cfg.bg[k];
    a.chunk = ctx->chunk;
    a.npack = (float *)ctx->npack.p;
    a.cmask = (uint32_t *)ctx->cmask.p;
    a.npack_stride = raster_npack_stride(d->color_mode, d->n_c, d->n_sigma);
    a.wait_status = (int *)((char *)ctx->small.p + kSmallFlags) + 1;
}

extern "C" {

snp_status snp_get_net_layout(const snp_scene_desc *desc, snp_net_layout *out)
{
    if (!desc || !out) return SNP_ERR_INVALID_ARG;
    const snp_status s = check_desc(nullptr, desc);
    if (s != SNP_OK) return s;
    layout_of(*desc, *out);
    return SNP_OK;
}

snp_status snp_default_chunks(const snp_scene_desc *desc, int32_t tile_size, int32_t *fwd_chunk, int32_t *bwd_chunk)
{
    if (!desc || !fwd_chunk || !bwd_chunk) return SNP_ERR_INVALID_ARG;
    const snp_status s = check_desc(nullptr, desc);
    if (s != SNP_OK) return s;
    const int ts = tile_size == 0 ? 16 : tile_size;
    if (ts != 8 && ts != 16 && ts != 32) return SNP_ERR_UNSUPPORTED;
    const bool dyn = desc->dynamic != 0;
    *fwd_chunk = raster_default_chunk(desc->color_mode, desc->n_c, desc->n_sigma, false, ts, dyn);
    *bwd_chunk = raster_default_chunk(desc->color_mode, desc->n_c, desc->n_sigma, true, ts, dyn);
    return SNP_OK;
}

snp_status snp_create(int32_t device, snp_context **out)
{
    if (!out) return SNP_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SNP_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return SNP_ERR_CUDA;
    snp_context *ctx = new snp_context();
    ctx->device = device;
    if (cudaMallocHost((void **)&ctx->h_views, sizeof(View) * kMaxViews) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_small, 64) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_views, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&ctx->loss_part.p, kLossSlots * 8 + 16) != cudaSuccess ||
        cudaMemset(ctx->loss_part.p, 0, kLossSlots * 8 + 16) != cudaSuccess) {
        snp_destroy(ctx);
        return SNP_ERR_CUDA;
    }
    ctx->loss_part.bytes = kLossSlots * 8 + 16;
    *out = ctx;
    return SNP_OK;
}

void snp_destroy(snp_context *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    Buf *bufs[] = {&ctx->views, &ctx->rec, &ctx->trect, &ctx->counts, &ctx->offsets, &ctx->scan_tmp, &ctx->keys,
                   &ctx->vals, &ctx->keys_alt, &ctx->vals_alt, &ctx->hist, &ctx->hist_scan, &ctx->ranges,
                   &ctx->px_state, &ctx->px_nwalk, &ctx->stats, &ctx->small, &ctx->g_view, &ctx->g_h0,
                   &ctx->qkeys, &ctx->qvals, &ctx->qkeys_alt, &ctx->qvals_alt, &ctx->qhist, &ctx->qhist_scan,
                   &ctx->npack, &ctx->cmask, &ctx->loss_part, &ctx->pop_cnt, &ctx->pop_tmp, &ctx->pop_total,
                   &ctx->colstore, &ctx->key_off};
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->h_views) cudaFreeHost(ctx->h_views);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    if (ctx->ev_views) cudaEventDestroy(ctx->ev_views);
    ctx->timer.destroy();
    delete ctx;
}

const char *snp_last_error(const snp_context *ctx) { return ctx ? ctx->err : "null context"; }

static snp_status ensure_keys(snp_context *ctx, int64_t K, int ts)
{
    ENS(keys, (size_t)K * 8);
    ENS(cmask, (size_t)K * (ts * ts / 32) * 4);
    ENS(key_off, (size_t)K * 4);
    ENS(keys_alt, (size_t)K * 8);
    ENS(vals, (size_t)K * 4);
    ENS(vals_alt, (size_t)K * 4);
    const int64_t hw = sort_hist_words(K);
    ENS(hist, (size_t)hw * 4);
    ENS(hist_scan, (size_t)hw * 4);
    return SNP_OK;
}

static snp_status ensure_frame(snp_context *ctx, int64_t n, int n_views, int64_t tiles, int64_t pixels,
                               const snp_scene_desc *d)
{
    const int64_t vn = n * n_views;
    ENS(views, sizeof(View) * kMaxViews);
    ENS(rec, (size_t)vn * kRecFloats * 4);
    ENS(trect, (size_t)vn * 16);
    ENS(counts, (size_t)vn * 4);
    ENS(offsets, (size_t)vn * 4);
    ENS(ranges, (size_t)tiles * 8);
    ENS(px_state, (size_t)pixels * 16);
    ENS(px_nwalk, (size_t)pixels * 4);
    ENS(stats, 64);
    ENS(small, kSmallBytes);
    ENS(qkeys, (size_t)tiles * 8);
    ENS(qkeys_alt, (size_t)tiles * 8);
    ENS(qvals, (size_t)tiles * 4);
    ENS(qvals_alt, (size_t)tiles * 4);
    ENS(qhist, (size_t)sort_hist_words(tiles) * 4);
    ENS(qhist_scan, (size_t)sort_hist_words(tiles) * 4);
    ENS(npack, (size_t)n * raster_npack_stride(d->color_mode, d->n_c, d->n_sigma) * 4);
    return SNP_OK;
}

// Bytes per composited pair of the forward's store: (colour, alpha_hat) with a
// colour network, alpha_hat alone otherwise.
static size_t store_pair_bytes(const snp_scene_desc *d) { return d->color_mode == SNP_COLOR_MLP ? 16 : 4; }

// Colour-store capacity (pairs) for K keys: the previous forward's composited count
// plus a quarter, else 16 per key, plus the partly used blocks of the forward CTAs;
// at most every (key, pixel) pair and 2^32 - 2.
static int64_t col_pairs_wanted(const snp_context *ctx, int64_t K, int ts)
{
    int64_t want = ctx->last_comp > 0 ? ctx->last_comp + ctx->last_comp / 4 : K * 16;
    // up to four forward CTAs per SM each hold one partly used block
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || sms <= 0)
        sms = 1024;
    want += (int64_t)4 * sms * kColBlock;
    want = std::max<int64_t>(want, (int64_t)1 << 16);
    want = std::min<int64_t>(want, std::max<int64_t>(K, 1) * ts * ts);
    return std::min<int64_t>(want, (int64_t)0xfffffffe);
}

static snp_status ensure_scan_tmp(snp_context *ctx, int64_t vn, int64_t key_bound, int64_t tiles)
{
    int64_t w = scan_temp_words(vn);
    const int64_t hw = scan_temp_words(sort_hist_words(key_bound));
    if (hw > w) w = hw;
    const int64_t tw = scan_temp_words(sort_hist_words(tiles));
    if (tw > w) w = tw;
    ENS(scan_tmp, (size_t)(w + 16) * 4);
    return SNP_OK;
}

snp_status snp_reserve(snp_context *ctx, const snp_scene_desc *desc, const snp_camera *cams, int32_t n_cams,
                       const snp_config *cfg, int64_t max_keys)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    if ((s = check_cams(ctx, cams, n_cams)) != SNP_OK) return s;
    if ((s = check_instances(ctx, desc->n, n_cams)) != SNP_OK) return s;
    const int ts = cfg && cfg->tile_size ? cfg->tile_size : 16;
    if (ts != 8 && ts != 16 && ts != 32) return fail(ctx, SNP_ERR_UNSUPPORTED, "tile_size %d not built", ts);
    if (max_keys <= 0) max_keys = std::min<int64_t>(4 * desc->n * n_cams + 1024, (int64_t)0xffffffff);
    if (max_keys > (int64_t)0xffffffff)
        return fail(ctx, SNP_ERR_UNSUPPORTED, "max_keys %lld exceeds 2^32 - 1", (long long)max_keys);
    int64_t tiles, pixels;
    ctx->reserved = false;
    if ((s = build_views(ctx, cams, n_cams, ts, &tiles, &pixels)) != SNP_OK) return s;
    if ((s = ensure_frame(ctx, desc->n, n_cams, tiles, pixels, desc)) != SNP_OK) return s;
    if ((s = ensure_keys(ctx, max_keys, ts)) != SNP_OK) return s;
    if ((s = ensure_scan_tmp(ctx, desc->n * n_cams, max_keys, tiles)) != SNP_OK) return s;
    // the view table of the reserved cameras stays on the device for captured forwards
    CK(cudaMemcpy(ctx->views.p, ctx->h_views, sizeof(View) * n_cams, cudaMemcpyHostToDevice));
    memcpy(ctx->res_cams, cams, sizeof(snp_camera) * n_cams);
    ctx->res_n_cams = n_cams;
    ctx->res_ts = ts;
    ctx->res_tiles = tiles;
    ctx->res_pixels = pixels;
    {
        const int nc = desc->color_mode == SNP_COLOR_MLP ? desc->n_c : 1;
        ENS(g_view, (size_t)desc->n * n_cams * kGvFloats * 4);
        ENS(g_h0, (size_t)desc->n * nc * 4);
    }
    if (!(cfg && (cfg->flags & SNP_FLAG_REPLAY_COLOR)))
        ENS(colstore, (size_t)col_pairs_wanted(ctx, max_keys, ts) * store_pair_bytes(desc));
    ctx->key_cap = max_keys;
    ctx->reserved = true;
    return SNP_OK;
}

snp_status snp_render_forward(snp_context *ctx, const snp_scene_desc *desc, const snp_scene_ptrs *scene,
                              const snp_camera *cams, int32_t n_cams, const snp_config *cfg, float *images,
                              int64_t *token, void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    if ((s = check_cams(ctx, cams, n_cams)) != SNP_OK) return s;
    if ((s = check_instances(ctx, desc->n, n_cams)) != SNP_OK) return s;
    if (!scene || !images || (desc->n > 0 && (!scene->geom || !scene->net)))
        return fail(ctx, SNP_ERR_INVALID_ARG, "null scene or image pointer");
    if (((uintptr_t)scene->geom & 15) || ((uintptr_t)scene->net & 15))
        return fail(ctx, SNP_ERR_INVALID_ARG, "scene arrays must be 16-byte aligned");
    snp_config c{};
    c.tile_size = 16;
    c.t_min = 1e-4f;
    if (cfg) c = *cfg;
    if (c.tile_size == 0) c.tile_size = 16;
    if (c.tile_size != 8 && c.tile_size != 16 && c.tile_size != 32)
        return fail(ctx, SNP_ERR_UNSUPPORTED, "tile_size %d not built", c.tile_size);
    if (c.integral_form != SNP_FORM_STABLE && c.integral_form != SNP_FORM_NAIVE)
        return fail(ctx, SNP_ERR_INVALID_ARG, "bad integral_form %d", c.integral_form);
    if (!(c.t_min >= 0.0f) || !(c.t_min < 1.0f)) return fail(ctx, SNP_ERR_INVALID_ARG, "t_min must be in [0, 1)");
    if (c.chunk < 0 || c.bwd_chunk < 0) return fail(ctx, SNP_ERR_INVALID_ARG, "negative chunk");
    const int ts = c.tile_size;
    const int chunk =
        c.chunk > 0 ? c.chunk : raster_default_chunk(desc->color_mode, desc->n_c, desc->n_sigma, false, ts, desc->dynamic != 0);
    if (chunk > 64 || raster_fwd_smem(desc->color_mode, desc->n_c, desc->n_sigma, chunk, ts) > 220 * 1024)
        return fail(ctx, SNP_ERR_INVALID_ARG, "chunk %d too large", chunk);

    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    int64_t tiles, pixels;
    if (capturing) {
        // no host synchronisation and no upload: use the reservation's device view table
        if (!ctx->reserved)
            return fail(ctx, SNP_ERR_INVALID_ARG, "a forward under stream capture needs snp_reserve first");
        if (n_cams != ctx->res_n_cams || memcmp(cams, ctx->res_cams, sizeof(snp_camera) * n_cams) != 0 ||
            ts != ctx->res_ts)
            return fail(ctx, SNP_ERR_INVALID_ARG, "a captured forward must use the reserved cameras and tile size");
        tiles = ctx->res_tiles;
        pixels = ctx->res_pixels;
    } else if ((s = build_views(ctx, cams, n_cams, ts, &tiles, &pixels)) != SNP_OK) {
        return s;
    }
    if (ctx->reserved && ts != ctx->res_ts)
        return fail(ctx, SNP_ERR_INVALID_ARG, "the context is reserved for tile size %d, not %d", ctx->res_ts, ts);
    const int64_t n = desc->n, vn = n * n_cams;
    if ((s = ensure_frame(ctx, n, n_cams, tiles, pixels, desc)) != SNP_OK) return s;
    ctx->token++;  // invalidates the previous forward's state from here on
    ctx->n_views = n_cams;
    ctx->n = n;
    ctx->n_tiles = tiles;
    ctx->n_pixels = pixels;
    ctx->desc = *desc;
    ctx->cfg = c;
    ctx->ts = ts;
    ctx->chunk = chunk;

    if (!capturing) {
        CK(cudaMemcpyAsync(ctx->views.p, ctx->h_views, sizeof(View) * n_cams, cudaMemcpyHostToDevice, st));
        CK(cudaEventRecord(ctx->ev_views, st));
    }
    uint32_t *d_total = (uint32_t *)((char *)ctx->small.p + kSmallTotal);
    int32_t *d_flags = (int32_t *)((char *)ctx->small.p + kSmallFlags);
    uint32_t *d_tiles = (uint32_t *)((char *)ctx->small.p + kSmallTiles);
    int *d_work = (int *)((char *)ctx->small.p + kSmallWork);

    int64_t key_bound;
    if (!ctx->reserved) {
        if ((s = ensure_scan_tmp(ctx, vn, 0, tiles)) != SNP_OK) return s;
    }
    ctx->timing = (c.flags & SNP_FLAG_STAGE_TIMING) != 0 && !capturing;
    STAGE_BEGIN(SNP_STAGE_PROJECT);
    launch_project((const float *)scene->geom, n, (const View *)ctx->views.p, n_cams, ts, (float *)ctx->rec.p,
                   (int4 *)ctx->trect.p, (uint32_t *)ctx->counts.p, st);
    {
        RasterArgs pa;
        fill_args(pa, ctx, desc, scene, nullptr);
        if ((s = launch_pack_net(pa, desc->color_mode, desc->n_c, desc->weight_dtype == SNP_BF16, st)) != SNP_OK) {
            STAGE_END();
            return fail(ctx, s, "network pack launch failed");
        }
        if (desc->color_mode == SNP_COLOR_SH) {
            snp_net_layout L;
            layout_of(*desc, L);
            launch_sh_color((const float *)scene->geom, scene->net, desc->weight_dtype == SNP_BF16, n,
                            (const View *)ctx->views.p, n_cams, L.off[11], L.off[13], L.stride, (float *)ctx->rec.p,
                            st);
        }
    }
    STAGE_END();
    STAGE_BEGIN(SNP_STAGE_SCAN);
    scan_u32((const uint32_t *)ctx->counts.p, (uint32_t *)ctx->offsets.p, vn, d_total, (uint32_t *)ctx->scan_tmp.p,
             st);
    STAGE_END();
    if (!ctx->reserved) {
        CK(cudaMemcpyAsync(ctx->h_small, d_total, 4, cudaMemcpyDeviceToHost, st));
        if (ctx->fwd_done)  // the previous forward's composited count sizes the colour store
            CK(cudaMemcpyAsync(ctx->h_small + 8, (char *)ctx->stats.p + 16, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (ctx->fwd_done) {
            uint64_t comp;
            memcpy(&comp, ctx->h_small + 8, 8);
            ctx->last_comp = (int64_t)comp;
        }
        key_bound = ctx->h_small[0];
        if ((s = ensure_keys(ctx, key_bound, ts)) != SNP_OK) return s;
        if ((s = ensure_scan_tmp(ctx, vn, key_bound, tiles)) != SNP_OK) return s;
        ctx->K = key_bound;
    } else {
        key_bound = ctx->key_cap;
        ctx->K = -1;  // known on the device only
    }
    CK(cudaMemsetAsync(d_flags, 0, 8, st));  // key overflow, device-wait timeout
    STAGE_BEGIN(SNP_STAGE_EMIT);
    launch_emit((const int4 *)ctx->trect.p, (const uint32_t *)ctx->counts.p, (const uint32_t *)ctx->offsets.p,
                (const float *)ctx->rec.p, n, (const View *)ctx->views.p, n_cams, (uint64_t *)ctx->keys.p,
                (uint32_t *)ctx->vals.p, key_bound, d_flags, st);
    uint32_t *d_nsort = (uint32_t *)((char *)ctx->small.p + kSmallNsort);
    launch_clamp_count(d_total, key_bound, d_nsort, st);
    STAGE_END();
    const int nbits = 32 + tile_bits(tiles);
    STAGE_BEGIN(SNP_STAGE_SORT);
    ctx->keys_in_alt = radix_sort((uint64_t *)ctx->keys.p, (uint32_t *)ctx->vals.p, (uint64_t *)ctx->keys_alt.p,
                                  (uint32_t *)ctx->vals_alt.p, d_nsort, key_bound, nbits, (uint32_t *)ctx->hist.p,
                                  (uint32_t *)ctx->hist_scan.p, (uint32_t *)ctx->scan_tmp.p, st);
    STAGE_END();
    const uint64_t *skeys = (const uint64_t *)(ctx->keys_in_alt ? ctx->keys_alt.p : ctx->keys.p);
    const uint32_t *svals = (const uint32_t *)(ctx->keys_in_alt ? ctx->vals_alt.p : ctx->vals.p);
    STAGE_BEGIN(SNP_STAGE_RANGES);
    CK(cudaMemsetAsync(ctx->ranges.p, 0, (size_t)tiles * 8, st));
    launch_tile_ranges(skeys, d_nsort, key_bound, (uint2 *)ctx->ranges.p, st);
    // persistent raster work queue: tiles by decreasing list length (on request)
    if (c.flags & SNP_FLAG_LENGTH_QUEUE) {
    launch_tile_queue((const uint2 *)ctx->ranges.p, tiles, (uint64_t *)ctx->qkeys.p, (uint32_t *)ctx->qvals.p,
                      d_tiles, st);
    ctx->queue_in_alt = radix_sort((uint64_t *)ctx->qkeys.p, (uint32_t *)ctx->qvals.p, (uint64_t *)ctx->qkeys_alt.p,
                                   (uint32_t *)ctx->qvals_alt.p, d_tiles, tiles, 32, (uint32_t *)ctx->qhist.p,
                                   (uint32_t *)ctx->qhist_scan.p, (uint32_t *)ctx->scan_tmp.p, st);
    }
    STAGE_END();
    CK(cudaMemsetAsync(ctx->stats.p, 0, 24, st));

    RasterArgs a;
    fill_args(a, ctx, desc, scene, svals);
    a.image = images;
    a.px_state = (float4 *)ctx->px_state.p;
    a.px_nwalk = (uint32_t *)ctx->px_nwalk.p;
    a.stats = (unsigned long long *)ctx->stats.p;
    a.work_counter = d_work;
    a.queue = (c.flags & SNP_FLAG_LENGTH_QUEUE)
                  ? (const uint32_t *)(ctx->queue_in_alt ? ctx->qvals_alt.p : ctx->qvals.p)
                  : nullptr;
    CK(cudaMemsetAsync(d_work, 0, 4, st));
    const size_t spb = store_pair_bytes(desc);
    ctx->col_on = !(c.flags & SNP_FLAG_REPLAY_COLOR);
    if (ctx->col_on && !ctx->reserved &&
        ensure(ctx, ctx->colstore, (size_t)col_pairs_wanted(ctx, key_bound, ts) * spb, "colstore") != SNP_OK) {
        // no room for the store: the backward recomputes the colours / alpha_hat instead
        cudaGetLastError();
        ctx->err[0] = 0;
        ctx->col_on = false;
    }
    if (ctx->col_on) ctx->col_on = ctx->colstore.bytes >= spb;
    if (ctx->col_on) {
        unsigned long long *d_col = (unsigned long long *)((char *)ctx->small.p + kSmallColCount);
        CK(cudaMemsetAsync(d_col, 0, 8, st));
        if (desc->color_mode == SNP_COLOR_MLP) a.colstore = (float4 *)ctx->colstore.p;
        else a.ahstore = (float *)ctx->colstore.p;
        a.key_off = (uint32_t *)ctx->key_off.p;
        a.col_count = d_col;
        a.col_cap = (uint32_t)std::min<size_t>(ctx->colstore.bytes / spb, (size_t)0xfffffffe);
        // test hook: SNP_TEST_COLSTORE_PAIRS caps the store, so that tests can drive the
        // backward's per-chunk recomputation of the pairs that did not fit
        if (const char *cap_env = getenv("SNP_TEST_COLSTORE_PAIRS")) {
            const long long v = atoll(cap_env);
            if (v >= 0 && (unsigned long long)v < a.col_cap) a.col_cap = (uint32_t)v;
        }
    }
    STAGE_BEGIN(SNP_STAGE_RASTER_FWD);
    note_raster_ctas(0);
    s = launch_raster_fwd(a, desc->color_mode, desc->n_c, c.integral_form, desc->weight_dtype == SNP_BF16, ts, st);
    if (s == SNP_OK) ctx->fwd_ctas = last_raster_ctas();
    STAGE_END();
    ctx->fwd_done = true;
    if (s != SNP_OK) return fail(ctx, s, "raster forward launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    CK(cudaGetLastError());
    if (token) *token = ctx->token;
    return SNP_OK;
}

snp_status snp_render_backward(snp_context *ctx, int64_t token, const snp_scene_desc *desc,
                               const snp_scene_ptrs *scene, const float *dL_dimages, const snp_grad_ptrs *grads,
                               void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    if (token != ctx->token || token == 0)
        return fail(ctx, SNP_ERR_INVALID_ARG, "stale token %lld (latest forward is %lld)", (long long)token,
                    (long long)ctx->token);
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    if (desc->n != ctx->desc.n || desc->n_sigma != ctx->desc.n_sigma || desc->color_mode != ctx->desc.color_mode ||
        desc->n_c != ctx->desc.n_c || desc->weight_dtype != ctx->desc.weight_dtype ||
        desc->dynamic != ctx->desc.dynamic || desc->omega0 != ctx->desc.omega0)
        return fail(ctx, SNP_ERR_INVALID_ARG, "scene description differs from the forward's");
    if (!scene || !dL_dimages || !grads || (desc->n > 0 && (!scene->geom || !scene->net)))
        return fail(ctx, SNP_ERR_INVALID_ARG, "null pointer");
    if ((((uintptr_t)scene->geom) | ((uintptr_t)scene->net) | ((uintptr_t)grads->net)) & 15u)
        return fail(ctx, SNP_ERR_INVALID_ARG, "scene arrays and the network gradient must be 16-byte aligned");
    if ((((uintptr_t)grads->geom) | ((uintptr_t)dL_dimages)) & 3u)
        return fail(ctx, SNP_ERR_INVALID_ARG, "the geometry gradient and dL/dimages must be 4-byte aligned");
    const int64_t n = desc->n, vn = n * ctx->n_views;
    const int nc = desc->color_mode == SNP_COLOR_MLP ? desc->n_c : 1;
    ENS(g_view, (size_t)vn * kGvFloats * 4);
    ENS(g_h0, (size_t)n * nc * 4);
    CK(cudaMemsetAsync(ctx->g_view.p, 0, (size_t)vn * kGvFloats * 4, st));
    CK(cudaMemsetAsync(ctx->g_h0.p, 0, (size_t)n * nc * 4, st));
    const uint32_t *svals = (const uint32_t *)(ctx->keys_in_alt ? ctx->vals_alt.p : ctx->vals.p);
    RasterArgs a;
    fill_args(a, ctx, desc, scene, svals);
    if (ctx->col_on) {
        if (desc->color_mode == SNP_COLOR_MLP) a.colstore = (float4 *)ctx->colstore.p;
        else a.ahstore = (float *)ctx->colstore.p;
        a.key_off = (uint32_t *)ctx->key_off.p;
    }
    a.px_state = (float4 *)ctx->px_state.p;
    a.px_nwalk = (uint32_t *)ctx->px_nwalk.p;
    a.dL_dimage = dL_dimages;
    a.g_net = grads->net;
    a.g_view = (float *)ctx->g_view.p;
    a.g_h0 = (float *)ctx->g_h0.p;
    a.chunk = raster_default_chunk(desc->color_mode, desc->n_c, desc->n_sigma, true, ctx->ts, desc->dynamic != 0);
    if (ctx->cfg.bwd_chunk > 0 && ctx->cfg.bwd_chunk < a.chunk) a.chunk = ctx->cfg.bwd_chunk;
    // test hook: SNP_TEST_STUCK_WAIT=1 makes the tensor-memory backward (N_c = 64) run
    // one bounded wait out, so that tests can check that it is reported
    // (SNP_ERR_TIMEOUT from snp_get_stats) and that the context stays usable
    if (const char *sw = getenv("SNP_TEST_STUCK_WAIT")) a.test_stuck_wait = atoi(sw) != 0;
    int *d_work = (int *)((char *)ctx->small.p + kSmallWork);
    a.work_counter = d_work;
    a.queue = (ctx->cfg.flags & SNP_FLAG_LENGTH_QUEUE)
                  ? (const uint32_t *)(ctx->queue_in_alt ? ctx->qvals_alt.p : ctx->qvals.p)
                  : nullptr;
    CK(cudaMemsetAsync(d_work, 0, 4, st));
    STAGE_BEGIN(SNP_STAGE_RASTER_BWD);
    note_raster_ctas(0);
    s = launch_raster_bwd(a, desc->color_mode, desc->n_c, ctx->cfg.integral_form, desc->weight_dtype == SNP_BF16,
                          ctx->ts, st);
    STAGE_END();
    if (s != SNP_OK) return fail(ctx, s, "raster backward launch failed");
    ctx->bwd_ctas = last_raster_ctas();
    STAGE_BEGIN(SNP_STAGE_POST_BWD);
    if (grads->geom)
        launch_project_bwd((const float *)scene->geom, n, (const View *)ctx->views.p, ctx->n_views,
                           (const float *)ctx->g_view.p, desc->color_mode == SNP_COLOR_CONST, grads->geom, st);
    if (desc->color_mode == SNP_COLOR_SH && (grads->geom || grads->net)) {
        snp_net_layout L;
        layout_of(*desc, L);
        launch_sh_bwd((const float *)scene->geom, scene->net, desc->weight_dtype == SNP_BF16, n,
                      (const View *)ctx->views.p, ctx->n_views, L.off[11], L.off[13], L.stride,
                      (const float *)ctx->rec.p, (const float *)ctx->g_view.p, grads->net, grads->geom, st);
    }
    if (grads->net && desc->color_mode == SNP_COLOR_MLP)
        launch_color_post(scene->net, desc->weight_dtype == SNP_BF16, n, desc->n_c, a.off_feat, a.off_Wc1,
                          a.off_bc1, a.stride, (const float *)ctx->g_h0.p, grads->net, st);
    STAGE_END();
    CK(cudaGetLastError());
    return SNP_OK;
}

}  // extern "C"

__global__ void k_fill_f32(float *p, int64_t n, float v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

extern "C" {

snp_status snp_autotune(snp_context *ctx, const snp_scene_desc *desc, const snp_scene_ptrs *scene,
                        const snp_camera *cams, int32_t n_cams, const snp_config *base, int32_t with_backward,
                        snp_config *best, float *best_ms, void *stream)
{
    if (!ctx || !desc || !scene || !cams || !best || !best_ms) return SNP_ERR_INVALID_ARG;
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    if ((s = check_cams(ctx, cams, n_cams)) != SNP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    snp_config b{};
    b.t_min = 1e-4f;
    if (base) b = *base;
    b.flags &= ~SNP_FLAG_STAGE_TIMING;
    int64_t pixels = 0;
    for (int v = 0; v < n_cams; ++v) pixels += (int64_t)cams[v].width * cams[v].height;
    snp_net_layout L;
    layout_of(*desc, L);
    float *img = nullptr, *dL = nullptr, *gg = nullptr, *gn = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (img) cudaFree(img);
        if (dL) cudaFree(dL);
        if (gg) cudaFree(gg);
        if (gn) cudaFree(gn);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&img, (size_t)pixels * 12 + 16) != cudaSuccess ||
        cudaMalloc(&dL, (size_t)pixels * 12 + 16) != cudaSuccess ||
        (with_backward && cudaMalloc(&gg, (size_t)desc->n * SNP_GEOM_STRIDE * 4 + 16) != cudaSuccess) ||
        (with_backward && cudaMalloc(&gn, (size_t)desc->n * L.stride * 4 + 16) != cudaSuccess) ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return fail(ctx, SNP_ERR_CUDA, "autotune: allocation failed");
    }
    k_fill_f32<<<(unsigned)((pixels * 3 + 255) / 256), 256, 0, st>>>(dL, pixels * 3, 1e-3f);
    note_launch();
    snp_grad_ptrs gp{gg, gn};
    float best_t = 1e30f;
    snp_config best_c = b;
    const int sizes[3] = {8, 16, 32};
    for (int ti = 0; ti < 3; ++ti) {
        const int ts = sizes[ti];
        const int dch = raster_default_chunk(desc->color_mode, desc->n_c, desc->n_sigma, false, ts, desc->dynamic != 0);
        const int chunks[2] = {dch, dch / 2 > 0 ? dch / 2 : 1};
        for (int ci = 0; ci < (chunks[1] == chunks[0] ? 1 : 2); ++ci) {
            snp_config c = b;
            c.tile_size = ts;
            c.chunk = chunks[ci];
            float t = 0.0f;
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                int64_t tok = 0;
                if (rep == 1) cudaEventRecord(e0, st);
                ok = snp_render_forward(ctx, desc, scene, cams, n_cams, &c, img, &tok, stream) == SNP_OK;
                if (ok && with_backward) ok = snp_render_backward(ctx, tok, desc, scene, dL, &gp, stream) == SNP_OK;
            }
            if (!ok) continue;  // e.g. a chunk the shared memory cannot hold
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cleanup();
                return fail(ctx, SNP_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
            }
            cudaEventElapsedTime(&t, e0, e1);
            t *= 0.5f;
            if (t < best_t) {
                best_t = t;
                best_c = c;
            }
        }
    }
    cleanup();
    if (best_t >= 1e30f) return fail(ctx, SNP_ERR_UNSUPPORTED, "autotune: no configuration ran");
    *best = best_c;
    *best_ms = best_t;
    return SNP_OK;
}

snp_status snp_stage_times(snp_context *ctx, double *ms, int64_t *calls, int32_t reset)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    CK(cudaSetDevice(ctx->device));
    ctx->timer.collect();
    for (int k = 0; k < SNP_N_STAGES; ++k) {
        if (ms) ms[k] = ctx->timer.ms[k];
        if (calls) calls[k] = ctx->timer.calls[k];
        if (reset) {
            ctx->timer.ms[k] = 0.0;
            ctx->timer.calls[k] = 0;
        }
    }
    return SNP_OK;
}

int64_t snp_kernel_launches(void) { return (int64_t)g_launches.load(); }

snp_status snp_mse_loss(snp_context *ctx, const float *image, const float *target, int64_t n, float *dL_dimage,
                        float *loss, void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 0) return fail(ctx, SNP_ERR_INVALID_ARG, "negative value count %lld", (long long)n);
    if (!loss || (n > 0 && (!image || !target || !dL_dimage))) return fail(ctx, SNP_ERR_INVALID_ARG, "null pointer");
    CK(cudaSetDevice(ctx->device));
    if (n == 0) {
        CK(cudaMemsetAsync(loss, 0, sizeof(float), st));
        return SNP_OK;
    }
    double *part = (double *)ctx->loss_part.p;
    unsigned *counter = (unsigned *)(part + kLossSlots);
    const snp_status s = launch_mse_loss(image, target, n, dL_dimage, loss, part, counter, kLossSlots, st);
    if (s != SNP_OK) return fail(ctx, s, "loss launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return SNP_OK;
}

snp_status snp_get_stats(snp_context *ctx, int64_t token, snp_stats *out, void *stream)
{
    if (!ctx || !out) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (token != ctx->token || token == 0) return fail(ctx, SNP_ERR_INVALID_ARG, "stale token");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long h[3];
    CK(cudaMemcpyAsync(h, ctx->stats.p, 24, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_small, ctx->small.p, 32, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out->n_keys = ctx->h_small[0];
    out->n_tiles = ctx->n_tiles;
    out->n_pixels = ctx->n_pixels;
    out->n_candidates = (int64_t)h[0];
    out->n_hits = (int64_t)h[1];
    out->n_composited = (int64_t)h[2];
    out->fwd_ctas_per_sm = ctx->fwd_ctas;
    out->bwd_ctas_per_sm = ctx->bwd_ctas;
    if (ctx->h_small[4] != 0) return fail(ctx, SNP_ERR_CAPACITY, "tile keys exceeded the reserved capacity");
    if (ctx->h_small[5] != 0) return fail(ctx, SNP_ERR_TIMEOUT, "a bounded device wait of the backward gave up");
    return SNP_OK;
}

snp_status snp_debug_keys(snp_context *ctx, int64_t token, uint64_t *keys_host, uint32_t *vals_host, int64_t cap,
                          int64_t *k_out, void *stream)
{
    if (!ctx || !k_out) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (token != ctx->token || token == 0) return fail(ctx, SNP_ERR_INVALID_ARG, "stale token");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ctx->h_small, ctx->small.p, 32, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int64_t K = ctx->h_small[0];
    *k_out = K;
    if (ctx->h_small[4] != 0) return fail(ctx, SNP_ERR_CAPACITY, "tile keys exceeded the reserved capacity");
    if (!keys_host && !vals_host) return SNP_OK;  // size query
    if (K > cap) return fail(ctx, SNP_ERR_INVALID_ARG, "host capacity %lld < K %lld", (long long)cap, (long long)K);
    if (K > 0) {
        const void *kp = ctx->keys_in_alt ? ctx->keys_alt.p : ctx->keys.p;
        const void *vp = ctx->keys_in_alt ? ctx->vals_alt.p : ctx->vals.p;
        if (keys_host) CK(cudaMemcpyAsync(keys_host, kp, (size_t)K * 8, cudaMemcpyDeviceToHost, st));
        if (vals_host) CK(cudaMemcpyAsync(vals_host, vp, (size_t)K * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return SNP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ training-step services

// Growth of the population-control scratch: an offline call, allowed on a
// reserved context too (it synchronises anyway).
static snp_status ensure_offline(snp_context *ctx, Buf &b, size_t bytes, const char *name)
{
    const bool r = ctx->reserved;
    ctx->reserved = false;
    const snp_status s = ensure(ctx, b, bytes, name);
    ctx->reserved = r;
    return s;
}

snp_status snp_popctl_accumulate(snp_context *ctx, const snp_scene_desc *desc, const float *g_net, float *stat_sum,
                                 int32_t *stat_count, void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    const int64_t n = desc->n;
    if (n > 0 && (!g_net || !stat_sum || !stat_count)) return fail(ctx, SNP_ERR_INVALID_ARG, "null pointer");
    CK(cudaSetDevice(ctx->device));
    snp_net_layout L;
    layout_of(*desc, L);
    PopFields f{};
    const int ns = desc->n_sigma;
    const int sizes[5] = {3 * ns, ns, ns, 1, ns};
    const int idx[5] = {0, 1, 2, 3, 12};
    for (int k = 0; k < 5; ++k)
        if (L.off[idx[k]] >= 0) {
            f.off[f.count] = L.off[idx[k]];
            f.size[f.count] = sizes[k];
            ++f.count;
        }
    f.stride = L.stride;
    if ((s = launch_popctl_stat(g_net, n, f, stat_sum, stat_count, (cudaStream_t)stream)) != SNP_OK)
        return fail(ctx, s, "statistic launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return SNP_OK;
}

snp_status snp_popctl_plan(snp_context *ctx, const snp_scene_desc *desc, const float *geom, const float *stat_sum,
                           const int32_t *stat_count, const snp_popctl_config *cfg, int32_t *action,
                           uint32_t *out_offset, int64_t *n_out, void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    const int64_t n = desc->n;
    if (!cfg || !n_out || (n > 0 && (!geom || !stat_sum || !stat_count || !action || !out_offset)))
        return fail(ctx, SNP_ERR_INVALID_ARG, "null pointer");
    if (!(cfg->extent > 0.0f) || !(cfg->grow_scale > 0.0f) || !(cfg->prune_scale > 0.0f))
        return fail(ctx, SNP_ERR_INVALID_ARG, "extent, grow_scale and prune_scale must be > 0");
    *n_out = 0;
    if (n == 0) return SNP_OK;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = ensure_offline(ctx, ctx->pop_cnt, (size_t)n * 4, "pop_cnt")) != SNP_OK) return s;
    if ((s = ensure_offline(ctx, ctx->pop_tmp, (size_t)scan_temp_words(n) * 4, "pop_tmp")) != SNP_OK) return s;
    if ((s = ensure_offline(ctx, ctx->pop_total, 16, "pop_total")) != SNP_OK) return s;
    PopThresholds t;
    t.grad = cfg->grad_threshold;
    t.prune = cfg->prune_threshold;
    t.log_grow = (float)log((double)cfg->grow_scale * (double)cfg->extent);
    t.log_prune = (float)log((double)cfg->prune_scale * (double)cfg->extent);
    if ((s = launch_popctl_plan(geom, n, stat_sum, stat_count, t, action, (uint32_t *)ctx->pop_cnt.p, st)) != SNP_OK)
        return fail(ctx, s, "plan launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    scan_u32((const uint32_t *)ctx->pop_cnt.p, out_offset, n, (uint32_t *)ctx->pop_total.p,
             (uint32_t *)ctx->pop_tmp.p, st);
    CK(cudaGetLastError());
    uint32_t total = 0;
    CK(cudaMemcpyAsync(&total, ctx->pop_total.p, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *n_out = total;
    return SNP_OK;
}

snp_status snp_popctl_apply(snp_context *ctx, const snp_scene_desc *desc, const snp_scene_ptrs *scene,
                            const int32_t *action, const uint32_t *out_offset, const float *noise, float *geom_out,
                            void *net_out, void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    const int64_t n = desc->n;
    if (n == 0) return SNP_OK;
    if (!scene || !scene->geom || !scene->net || !action || !out_offset || !noise || !geom_out || !net_out)
        return fail(ctx, SNP_ERR_INVALID_ARG, "null pointer");
    if ((((uintptr_t)scene->net) | ((uintptr_t)net_out)) & 15u)
        return fail(ctx, SNP_ERR_INVALID_ARG, "network arrays must be 16-byte aligned");
    CK(cudaSetDevice(ctx->device));
    snp_net_layout L;
    layout_of(*desc, L);
    const int row_bytes = L.stride * (desc->weight_dtype == SNP_BF16 ? 2 : 4);
    if ((s = launch_popctl_apply(scene->geom, scene->net, n, row_bytes, action, out_offset, noise,
                                 (float)log(1.6), geom_out, net_out, (cudaStream_t)stream)) != SNP_OK)
        return fail(ctx, s, "apply launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return SNP_OK;
}

snp_status snp_geom_reg(snp_context *ctx, const snp_scene_desc *desc, const float *geom, float weight,
                        float *g_geom, float *loss, void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    const int64_t n = desc->n;
    cudaStream_t st = (cudaStream_t)stream;
    if (!loss || (n > 0 && !geom)) return fail(ctx, SNP_ERR_INVALID_ARG, "null pointer");
    CK(cudaSetDevice(ctx->device));
    if (n == 0) {
        CK(cudaMemsetAsync(loss, 0, sizeof(float), st));
        return SNP_OK;
    }
    double *part = (double *)ctx->loss_part.p;
    unsigned *counter = (unsigned *)(part + kLossSlots);
    if ((s = launch_geom_reg(geom, n, (float)((double)weight / (double)n), g_geom, loss, part, counter, kLossSlots,
                             st)) != SNP_OK)
        return fail(ctx, s, "regulariser launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return SNP_OK;
}

snp_status snp_adam_step(snp_context *ctx, const snp_scene_desc *desc, float *geom, void *net, float *net_master,
                         const snp_grad_ptrs *grads, float *m_geom, float *v_geom, float *m_net, float *v_net,
                         const snp_adam_config *cfg, void *stream)
{
    if (!ctx) return SNP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    snp_status s;
    if ((s = check_desc(ctx, desc)) != SNP_OK) return s;
    if (!cfg || !grads) return fail(ctx, SNP_ERR_INVALID_ARG, "null pointer");
    if (cfg->step < 1) return fail(ctx, SNP_ERR_INVALID_ARG, "step must be >= 1, got %d", cfg->step);
    if (!(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
        !(cfg->eps > 0.0f))
        return fail(ctx, SNP_ERR_INVALID_ARG, "need 0 <= beta < 1 and eps > 0");
    const int64_t n = desc->n;
    if (n == 0) return SNP_OK;
    const bool bf16 = desc->weight_dtype == SNP_BF16;
    if (grads->geom && (!geom || !m_geom || !v_geom)) return fail(ctx, SNP_ERR_INVALID_ARG, "null geometry array");
    if (grads->net && (!net || !m_net || !v_net || (bf16 && !net_master)))
        return fail(ctx, SNP_ERR_INVALID_ARG, "null network array (BF16 weights need the FP32 master copy)");
    if (grads->net && ((((uintptr_t)net) | ((uintptr_t)grads->net) | ((uintptr_t)m_net) | ((uintptr_t)v_net) |
                        ((uintptr_t)(bf16 ? (void *)net_master : net))) & 15u))
        return fail(ctx, SNP_ERR_INVALID_ARG, "network arrays must be 16-byte aligned");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    AdamConsts c;
    c.beta1 = cfg->beta1;
    c.beta2 = cfg->beta2;
    c.one_m_beta1 = (float)(1.0 - (double)cfg->beta1);
    c.one_m_beta2 = (float)(1.0 - (double)cfg->beta2);
    c.corr1 = (float)(1.0 / (1.0 - pow((double)cfg->beta1, (double)cfg->step)));
    c.corr2 = (float)(1.0 / (1.0 - pow((double)cfg->beta2, (double)cfg->step)));
    c.eps = cfg->eps;
    if (grads->geom && (s = launch_adam_geom(geom, grads->geom, m_geom, v_geom, n, cfg->lr_geom, c, st)) != SNP_OK)
        return fail(ctx, s, "Adam launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (grads->net) {
        snp_net_layout L;
        layout_of(*desc, L);
        const int ns = desc->n_sigma, nc = desc->n_c;
        const int sizes[14] = {3 * ns, ns, ns, 1, kFeat, nc * (3 + kFeat), nc, nc * nc, nc, 3 * nc, 3, 48, ns, 36};
        AdamNetFields f;
        for (int k = 0; k < 14; ++k) {
            f.off[k] = L.off[k];
            f.end[k] = L.off[k] >= 0 ? L.off[k] + sizes[k] : -1;
            f.lr[k] = cfg->lr_net[k];
        }
        f.stride = L.stride;
        float *P = bf16 ? net_master : (float *)net;
        if ((s = launch_adam_net(P, bf16 ? net : nullptr, grads->net, m_net, v_net, n, f, c, st)) != SNP_OK)
            return fail(ctx, s, "Adam launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    return SNP_OK;
}
