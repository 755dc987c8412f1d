// snp_raster_fwd.cu -- forward per-tile rasterizer ("render kernel", App. A).
//
// One CTA per 16 x 16 screen tile.  The tile's depth-sorted list is walked in
// chunks staged in shared memory.  Each chunk runs in phases so that the
// expensive per-pair work is done by fully occupied warps:
//   P1 (one thread per pixel)   ray / ellipsoid test for every entry of the chunk,
//                               hits appended to per-entry pixel lists;
//   P2 (one thread per hit)     closed-form integral alpha_hat (Eq. 7/8);
//   P3 (one thread per pixel)   front-to-back compositing weights
//                               w = T (1 - exp(-alpha_hat)), T = exp(-sum alpha_hat)
//                               (Eq. 4, 9) and early termination -- transmittance
//                               does not depend on colour, so it is settled before
//                               any colour is evaluated; composited pairs are
//                               appended to per-entry lists;
//   P4 (one thread per pair)    colour MLP of every composited pair;
//   P5 (one thread per pixel)   C += w * colour in list order.
// The result is the sequential front-to-back composite.  The per-pixel
// composited colour, optical depth and number of list entries walked are saved
// for the backward pass.
#include "snp_raster.cuh"

namespace snp {

// Shared-memory footprint of the forward kernel for a chunk size.
static size_t fwd_smem_bytes(int nc, int ns, int chunk)
{
    const size_t per_entry = (size_t)entry_stride(ns, nc) * 4 + kRasterThreads * 4 /* alpha_hat */ +
                             kRasterThreads * 2 /* hit list */ +
                             (nc > 0 ? kRasterThreads * (4 + 12 + 2) /* w, colour, list */ : 0);
    return kRasterThreads * 16 /* rays */ + (size_t)chunk * per_entry;
}

template <int NC, int FORM, bool BF16>
__global__ void __launch_bounds__(kRasterThreads, 2) k_raster_fwd(RasterArgs a)
{
    extern __shared__ float4 smem4[];
    constexpr int NT = kRasterThreads;
    const int CH = a.chunk;
    const int ns = a.n_sigma;
    const int es = entry_stride(ns, NC);
    float4 *s_d = smem4;                                        // [NT] pixel rays
    float *sm = reinterpret_cast<float *>(smem4 + NT);          // [CH][es] staged entries
    float *s_ah = sm + CH * es;                                 // [CH][NT] alpha_hat
    float *s_w = s_ah + CH * NT;                                 // [CH][NT] weights (MLP)
    float *s_col = s_w + (NC > 0 ? CH * NT : 0);                // [3][CH][NT] colours (MLP)
    uint16_t *s_hl = reinterpret_cast<uint16_t *>(s_col + (NC > 0 ? 3 * CH * NT : 0));  // [CH][NT]
    uint16_t *s_al = s_hl + CH * NT;                            // [CH][NT] (MLP)
    __shared__ uint32_t s_gid[kMaxChunk];
    __shared__ int s_nh[65], s_na[65], s_ph[65], s_pa[65];
    __shared__ int s_view;

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    if (tid == 0) s_view = find_view(a.views, a.n_views, tile);
    __syncthreads();
    const int v = s_view;
    const View &V = a.views[v];
    const int lt = tile - V.tile_off;
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    int lx, ly;
    tile_pixel16(tid, lx, ly);
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const bool inside = px < V.width && py < V.height;
    const float3 d = pixel_ray(V, px, py);
    s_d[tid] = make_float4(d.x, d.y, d.z, 0.0f);
    const uint2 rg = a.ranges[tile];
    const int64_t vn = (int64_t)v * a.n;

    float3 C = make_float3(0.f, 0.f, 0.f);
    float tau = 0.0f, T = 1.0f;
    uint32_t nwalk = 0;
    bool alive = inside;
    uint32_t n_cand = 0, n_hit = 0, n_comp = 0;

    for (uint32_t c0 = rg.x; c0 < rg.y; c0 += CH) {
        const int cnt = min((int)(rg.y - c0), CH);
        __syncthreads();
        if (tid < cnt) {
            s_gid[tid] = a.vals[c0 + tid];
            s_nh[tid] = 0;
            s_na[tid] = 0;
        }
        __syncthreads();
        stage_chunk<NC, BF16>(sm, s_gid, cnt, vn, a, es);
        __syncthreads();

        // P1: which pixels' rays enter which ellipsoids
        for (int e = 0; e < cnt; ++e) {
            bool hit = false;
            if (alive) {
                ++n_cand;
                hit = hit_test(sm + e * es, d);
            }
            s_ah[e * NT + tid] = 0.0f;
            list_append(hit, (uint16_t)tid, &s_nh[e], s_hl + e * NT);
        }
        __syncthreads();
        if (tid < 32) warp_prefix64(s_nh, cnt, s_ph);
        __syncthreads();

        // P2: alpha_hat of every hit
        {
            const int nh = s_ph[cnt];
            int e = 0;
            for (int q = tid; q < nh; q += NT) {
                while (q >= s_ph[e + 1]) ++e;
                const int pix = s_hl[e * NT + (q - s_ph[e])];
                const float *R = sm + e * es;
                const float4 dd = s_d[pix];
                const float3 dv = make_float3(dd.x, dd.y, dd.z);
                Hit h;
                float ah = 0.0f;
                if (intersect(R, dv, h)) ah = integral<FORM>(R, R + kRecFloats, ns, dv, h);
                s_ah[e * NT + pix] = ah;
                ++n_hit;
            }
        }
        __syncthreads();

        // P3: compositing weights and termination, in list order
        for (int e = 0; e < cnt; ++e) {
            bool act = false;
            float w = 0.0f;
            if (alive) {
                const float ah = s_ah[e * NT + tid];
                if (ah > 0.0f) {
                    ++n_comp;
                    w = T * (1.0f - __expf(-ah));
                    tau += ah;
                    T = __expf(-tau);
                    nwalk = c0 - rg.x + e + 1;
                    act = true;
                    if constexpr (NC == 0) {
                        const float *R = sm + e * es;
                        C.x = fmaf(w, R[kRecRgb + 0], C.x);
                        C.y = fmaf(w, R[kRecRgb + 1], C.y);
                        C.z = fmaf(w, R[kRecRgb + 2], C.z);
                    }
                    if (T < a.t_min) alive = false;
                }
            }
            if constexpr (NC > 0) {
                s_w[e * NT + tid] = act ? w : -1.0f;
                list_append(act, (uint16_t)tid, &s_na[e], s_al + e * NT);
            }
        }

        if constexpr (NC > 0) {
            __syncthreads();
            if (tid < 32) warp_prefix64(s_na, cnt, s_pa);
            __syncthreads();
            // P4: colour of every composited pair
            const int na = s_pa[cnt];
            int e = 0;
            for (int q = tid; q < na; q += NT) {
                while (q >= s_pa[e + 1]) ++e;
                const int pix = s_al[e * NT + (q - s_pa[e])];
                const float4 dd = s_d[pix];
                const float3 col = mlp_color<NC>(sm + e * es + kRecFloats + den_stride(ns), make_float3(dd.x, dd.y, dd.z));
                s_col[(0 * CH + e) * NT + pix] = col.x;
                s_col[(1 * CH + e) * NT + pix] = col.y;
                s_col[(2 * CH + e) * NT + pix] = col.z;
            }
            __syncthreads();
            // P5: accumulate in list order
            for (int e2 = 0; e2 < cnt; ++e2) {
                const float w = s_w[e2 * NT + tid];
                if (w >= 0.0f) {
                    C.x = fmaf(w, s_col[(0 * CH + e2) * NT + tid], C.x);
                    C.y = fmaf(w, s_col[(1 * CH + e2) * NT + tid], C.y);
                    C.z = fmaf(w, s_col[(2 * CH + e2) * NT + tid], C.z);
                }
            }
        }
        if (__syncthreads_and(!alive)) break;
    }
    if (inside) {
        const int64_t p = V.pix_off + (int64_t)py * V.width + px;
        a.image[3 * p + 0] = fmaf(T, a.bg[0], C.x);
        a.image[3 * p + 1] = fmaf(T, a.bg[1], C.y);
        a.image[3 * p + 2] = fmaf(T, a.bg[2], C.z);
        if (a.px_state) {
            a.px_state[p] = make_float4(C.x, C.y, C.z, tau);
            a.px_nwalk[p] = nwalk;
        }
    }
    if (a.stats) {
        const unsigned long long s0 = warp_sum_u64(n_cand), s1 = warp_sum_u64(n_hit), s2 = warp_sum_u64(n_comp);
        if (lane_id() == 0) {
            atomicAdd(a.stats + 0, s0);
            atomicAdd(a.stats + 1, s1);
            atomicAdd(a.stats + 2, s2);
        }
    }
}

size_t raster_fwd_smem(int color_mode, int n_c, int n_sigma, int chunk)
{
    const int nc = color_mode == SNP_COLOR_MLP ? n_c : 0;
    return fwd_smem_bytes(nc, n_sigma, chunk);
}

int raster_default_chunk(int color_mode, int n_c, int n_sigma, bool backward)
{
    const int nc = color_mode == SNP_COLOR_MLP ? n_c : 0;
    if (backward) return raster_bwd_default_chunk(nc, n_sigma);
    int ch = 32;
    while (ch > 1 && fwd_smem_bytes(nc, n_sigma, ch) > 104 * 1024) --ch;
    return ch;
}

template <int NC, int FORM, bool BF16>
static snp_status run_fwd(const RasterArgs &a, cudaStream_t st)
{
    const size_t smem = fwd_smem_bytes(NC, a.n_sigma, a.chunk);
    if (smem > 220 * 1024 || a.chunk > 64) return SNP_ERR_INVALID_ARG;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_raster_fwd<NC, FORM, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr_set = true;
    }
    if (a.n_tiles <= 0) return SNP_OK;
    k_raster_fwd<NC, FORM, BF16><<<(unsigned)a.n_tiles, kRasterThreads, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}

template <int NC>
static snp_status dispatch_fwd(const RasterArgs &a, int form, int bf16, cudaStream_t st)
{
    if (form == SNP_FORM_STABLE)
        return bf16 ? run_fwd<NC, 0, true>(a, st) : run_fwd<NC, 0, false>(a, st);
    return bf16 ? run_fwd<NC, 1, true>(a, st) : run_fwd<NC, 1, false>(a, st);
}

snp_status launch_raster_fwd(const RasterArgs &a, int color_mode, int n_c, int form, int bf16, int ts,
                             cudaStream_t st)
{
    if (ts != 16) return SNP_ERR_UNSUPPORTED;
    if (color_mode == SNP_COLOR_CONST) return dispatch_fwd<0>(a, form, bf16, st);
    if (n_c == 32) return dispatch_fwd<32>(a, form, bf16, st);
    if (n_c == 64) return dispatch_fwd<64>(a, form, bf16, st);
    return SNP_ERR_UNSUPPORTED;
}

}  // namespace snp
