// snp_raster_fwd.cu -- forward per-tile rasterizer ("render kernel", App. A):
// one CTA per 16 x 16 screen tile, one thread per pixel.  The tile's depth-sorted
// list is walked in chunks staged in shared memory; every pixel intersects its
// ray with each ellipsoid, evaluates the closed-form integral (Eq. 8), the kernel
// alpha (Eq. 9) and the colour, and composites front to back (Eq. 4) until its
// transmittance drops below t_min.  The per-pixel composited colour, optical depth
// and number of list entries walked are saved for the backward pass.
#include "snp_raster.cuh"

namespace snp {

template <int NC, int FORM, bool BF16>
__global__ void __launch_bounds__(kRasterThreads) k_raster_fwd(RasterArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ uint32_t s_gid[kMaxChunk];
    __shared__ int s_view;

    const int tile = blockIdx.x;
    if (threadIdx.x == 0) s_view = find_view(a.views, a.n_views, tile);
    __syncthreads();
    const int v = s_view;
    const View &V = a.views[v];
    const int lt = tile - V.tile_off;
    const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
    int lx, ly;
    tile_pixel16(threadIdx.x, lx, ly);
    const int px = tx * 16 + lx, py = ty * 16 + ly;
    const bool inside = px < V.width && py < V.height;
    const float3 d = pixel_ray(V, px, py);
    const uint2 rg = a.ranges[tile];
    const int ns = a.n_sigma;
    const int es = entry_stride(ns, NC);
    const int64_t vn = (int64_t)v * a.n;

    float3 C = make_float3(0.f, 0.f, 0.f);
    float tau = 0.0f, T = 1.0f;
    uint32_t nwalk = 0;
    bool done = !inside;
    uint32_t n_cand = 0, n_hit = 0, n_comp = 0;

    for (uint32_t c0 = rg.x; c0 < rg.y; c0 += a.chunk) {
        const int cnt = min((int)(rg.y - c0), a.chunk);
        __syncthreads();
        if ((int)threadIdx.x < cnt) s_gid[threadIdx.x] = a.vals[c0 + threadIdx.x];
        __syncthreads();
        stage_chunk<NC, BF16>(sm, s_gid, cnt, vn, a, es);
        __syncthreads();
        if (!done) {
            for (int e = 0; e < cnt; ++e) {
                const float *R = sm + e * es;
                Hit h;
                ++n_cand;
                if (!intersect(R, d, h)) continue;
                ++n_hit;
                const float ah = integral<FORM>(R, R + kRecFloats, ns, d, h);
                if (!(ah > 0.0f)) continue;
                ++n_comp;
                float3 col;
                if constexpr (NC == 0)
                    col = make_float3(R[kRecRgb + 0], R[kRecRgb + 1], R[kRecRgb + 2]);
                else
                    col = mlp_color<NC>(R + kRecFloats + den_stride(ns), d);
                const float wgt = T * (1.0f - __expf(-ah));
                C.x = fmaf(wgt, col.x, C.x);
                C.y = fmaf(wgt, col.y, C.y);
                C.z = fmaf(wgt, col.z, C.z);
                tau += ah;
                T = __expf(-tau);
                nwalk = c0 - rg.x + e + 1;
                if (T < a.t_min) {
                    done = true;
                    break;
                }
            }
        }
        if (__syncthreads_and(done)) break;
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
    return (size_t)chunk * entry_stride(n_sigma, nc) * sizeof(float);
}

int raster_default_chunk(int color_mode, int n_c, int n_sigma, bool backward)
{
    const int nc = color_mode == SNP_COLOR_MLP ? n_c : 0;
    const int es = entry_stride(n_sigma, nc) * 4;
    const int budget = backward ? 48 * 1024 : 48 * 1024;
    int ch = budget / es;
    if (ch < 1) ch = 1;
    if (ch > 64) ch = 64;
    return ch;
}

template <int NC, int FORM, bool BF16>
static snp_status run_fwd(const RasterArgs &a, cudaStream_t st)
{
    const size_t smem = (size_t)a.chunk * entry_stride(a.n_sigma, NC) * sizeof(float);
    if (smem > 200 * 1024) return SNP_ERR_INVALID_ARG;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_raster_fwd<NC, FORM, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
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
