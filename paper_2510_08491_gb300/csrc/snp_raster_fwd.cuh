// snp_raster_fwd.cuh -- forward per-tile rasterizer ("render kernel", App. A).
//
// Persistent CTAs take screen tiles (of all views) from an atomic counter, in
// tile order or, on request, by decreasing list length.  A tile's depth-sorted
// list is walked in chunks staged in shared memory (cp.async copies of the
// projection records and the packed network blocks); each chunk runs in phases
// so that the expensive per-pair work is done by fully occupied warps:
//   P1 (per pixel)  ray / ellipsoid test for every entry of the chunk; hits are
//                   appended to per-entry pixel lists;
//   P2 (per hit)    closed-form integral alpha_hat (Eq. 7/8);
//   P3 (per pixel)  front-to-back weights w = T (1 - exp(-alpha_hat)),
//                   T = exp(-sum alpha_hat) (Eq. 4, 9) and early termination --
//                   transmittance does not depend on colour, so it is settled
//                   before any colour is evaluated; composited pairs are listed;
//   P4 (per warp)   colour MLP of the composited pairs in passes of 16 pairs of
//                   one list entry (tensor cores for the hidden layer);
//   P5 (per pixel)  C += w * colour in list order; with the colour store on, each
//                   composited pair's (colour, alpha_hat) is written to the key's
//                   slice of the store at the rank of its pixel among the key's
//                   composited pixels (the backward reads it back by the same rank).
// The result is the sequential front-to-back composite.  The per-pixel composited
// colour, optical depth, number of list entries walked and, per (tile, entry), the
// mask of pixels that composited it are saved for the backward pass.
#pragma once

#include "snp_raster.cuh"

namespace snp {

template <int TS>
__host__ __device__ inline size_t fwd_smem_bytes(int nc, int ns, int chunk)
{
    constexpr int NPIX = TileCfg<TS>::NPIX;
    const size_t per_entry = (size_t)entry_stride(ns, nc) * 4 + NPIX * 4 /* alpha_hat */ + NPIX * 2 /* hit list */ +
                             (nc > 0 ? NPIX * (4 + 12 + 2) /* weight, colour, list */ : 0) +
                             (NPIX / 32 + 1) * 4 /* mask words, store offset */;
    return NPIX * 32 /* rays */ + (size_t)chunk * per_entry;
}

// One warp: the chunk's slice of the forward's store (colour store, or alpha_hat
// store without a colour network), split by entry in list order (count[e] pairs
// each), taken from the CTA's current block or a new block of the global bump
// allocator; a chunk that does not fit gets kNoStore and the backward recomputes
// it.  Writes koff[e] and the keys' global offsets.
__device__ __forceinline__ void store_slices(const RasterArgs &a, const int *count, int cnt, uint32_t c0, int *pc,
                                             uint32_t *koff, unsigned long long &cbase, unsigned long long &blk_next,
                                             unsigned long long &blk_end)
{
    const int lane = threadIdx.x & 31;
    warp_prefix64(count, cnt, pc);
    __syncwarp();
    if (lane == 0) {
        const unsigned long long tot = (unsigned long long)pc[cnt];
        if (blk_next + tot > blk_end) {
            // a new block of the store for this CTA (the rest of the old one is left unused)
            const unsigned long long want = tot > kColBlock ? tot : kColBlock;
            const unsigned long long b = atomicAdd(a.col_count, want);
            const bool fits = b + want <= (unsigned long long)a.col_cap;
            blk_next = fits ? b : 0ull;
            blk_end = fits ? b + want : 0ull;
        }
        if (blk_next + tot <= blk_end) {
            cbase = blk_next;
            blk_next += tot;
        } else {
            cbase = ~0ull;  // store full: the backward recomputes this chunk
        }
    }
    __syncwarp();
    for (int ei = lane; ei < cnt; ei += 32) {
        const uint32_t o = cbase == ~0ull ? kNoStore : (uint32_t)(cbase + pc[ei]);
        koff[ei] = o;
        a.key_off[c0 + ei] = o;
    }
}

// One warp: per-entry composited counts of a chunk (cnt entries) from its masks,
// then the chunk's slice of the alpha_hat store.
template <int NPIX>
__device__ __forceinline__ void ahstore_slices(const RasterArgs &a, const uint32_t *cw, int cnt, uint32_t c0,
                                                 int *count, int *pc, uint32_t *koff, unsigned long long &cbase,
                                                 unsigned long long &blk_next, unsigned long long &blk_end)
{
    for (int e = threadIdx.x & 31; e < cnt; e += 32) {
        int c = 0;
        for (int w = 0; w < NPIX / 32; ++w) c += __popc(cw[e * (NPIX / 32) + w]);
        count[e] = c;
    }
    __syncwarp();
    store_slices(a, count, cnt, c0, pc, koff, cbase, blk_next, blk_end);
}

// Each thread writes alpha_hat of its pixels' composited pairs of a chunk (bit e of
// m[k]: pixel k composited entry e) at their ranks in the entries' store slices.
template <int NPIX, int NT, int PPT>
__device__ __forceinline__ void ahstore_write(const RasterArgs &a, const uint64_t (&m)[PPT], const uint32_t *koff,
                                              const uint32_t *cw, const float *s_ah, int tid)
{
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int slot = k * NT + tid;
        for (uint64_t mm = m[k]; mm != 0ull; mm &= mm - 1ull) {
            const int e = __ffsll((long long)mm) - 1;
            const uint32_t o = koff[e];
            if (o != kNoStore) a.ahstore[o + mask_rank<NPIX>(cw + e * (NPIX / 32), slot)] = s_ah[e * NPIX + slot];
        }
    }
}

template <int TS, int NC, int FORM, bool BF16>
__global__ void __launch_bounds__(TileCfg<TS>::NT, fwd_min_blocks(TS, NC)) k_raster_fwd(RasterArgs a)
{
    constexpr int NT = TileCfg<TS>::NT;
    constexpr int NPIX = TileCfg<TS>::NPIX;
    constexpr int PPT = TileCfg<TS>::PPT;
    extern __shared__ float4 smem4[];
    const int CH = a.chunk;
    const int ns = a.n_sigma;
    const int es = entry_stride(ns, NC);
    float4 *s_ray = smem4;                                      // [2 NPIX] pixel rays
    float *sm = reinterpret_cast<float *>(smem4 + 2 * NPIX);    // [CH][es] staged entries
    float *s_ah = sm + CH * es;                                 // [CH][NPIX] alpha_hat
    float *s_w = s_ah + CH * NPIX;                              // [CH][NPIX] weights (MLP)
    float *s_col = s_w + (NC > 0 ? CH * NPIX : 0);              // [3][CH][NPIX] colours (MLP)
    uint16_t *s_hl = reinterpret_cast<uint16_t *>(s_col + (NC > 0 ? 3 * CH * NPIX : 0));  // [CH][NPIX]
    uint16_t *s_al = s_hl + CH * NPIX;                          // [CH][NPIX] (MLP)
    uint32_t *s_cw = reinterpret_cast<uint32_t *>(s_al + (NC > 0 ? CH * NPIX : 0));  // [CH][NPIX/32] masks
    uint32_t *s_koff = s_cw + CH * (NPIX / 32);                  // [CH] store offsets
    __shared__ uint32_t s_gid[kMaxChunk];
    __shared__ int s_pc[65];
    __shared__ unsigned long long s_cbase, s_blk_next, s_blk_end;  // colour store: chunk base, CTA block
    __shared__ int s_nh[65], s_na[65], s_ph[65], s_nb[65], s_pb[65];
    __shared__ int s_view, s_item;

    const int tid = threadIdx.x;
    uint32_t n_cand = 0, n_hit = 0, n_comp = 0;
    if (tid == 0) s_blk_next = s_blk_end = 0;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_tiles) break;
        const int tile = a.queue ? (int)a.queue[item] : item;
        if (tid == 0) s_view = find_view(a.views, a.n_views, tile);
        __syncthreads();
        const int v = s_view;
        const View &V = a.views[v];
        const int lt = tile - V.tile_off;
        const int tx = lt % V.tiles_x, ty = lt / V.tiles_x;
        const CamK ck = cam_consts(V);
        int px[PPT], py[PPT];
        bool inside[PPT], alive[PPT];
        PixRay ry[PPT];
        float3 C[PPT];
        float tau[PPT], T[PPT];
        uint32_t nwalk[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            int lx, ly;
            tile_pixel<TS>(tid, k, lx, ly);
            px[k] = tx * TS + lx;
            py[k] = ty * TS + ly;
            inside[k] = px[k] < V.width && py[k] < V.height;
            ry[k] = pixel_ray(V, px[k], py[k]);
            store_ray(s_ray, k * NT + tid, ry[k]);
            alive[k] = inside[k];
            C[k] = make_float3(0.f, 0.f, 0.f);
            tau[k] = 0.0f;
            T[k] = 1.0f;
            nwalk[k] = 0;
        }
        const uint2 rg = a.ranges[tile];
        const int64_t vn = (int64_t)v * a.n;
        // alpha_hat store (no colour network): the chunk whose writes are still to be made
        bool pend = false;
        uint32_t pend_c0 = 0;
        int pend_cnt = 0;
        uint64_t pend_m[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) pend_m[k] = 0ull;

        // The chunk's record ids live in one half of s_gid; with a colour network the
        // next chunk's are copied into the other half (4-byte cp.async) from P2 on.
        bool pre = false;
        int ci = 0;
        for (uint32_t c0 = rg.x; c0 < rg.y; c0 += CH, ++ci) {
            const int cnt = min((int)(rg.y - c0), CH);
            uint32_t *const cg = s_gid + (NC > 0 ? (ci & 1) * (kMaxChunk / 2) : 0);
            __syncthreads();
            if (tid < cnt) {
                if (!pre) cg[tid] = a.vals[c0 + tid];
                s_nh[tid] = 0;
                s_na[tid] = 0;
            }
            if constexpr (NC == 0) {
                if (pend && tid < 32) ahstore_slices<NPIX>(a, s_cw, pend_cnt, pend_c0, s_nb, s_pc, s_koff, s_cbase, s_blk_next,
                                                    s_blk_end);
            }
            if (pre) cp_async_wait_all();
            __syncthreads();
            stage_chunk<NC, BF16>(sm, cg, cnt, vn, a, es, V.time);
            __syncthreads();
            if constexpr (NC == 0) {
                // the previous chunk's alpha_hat before P1 clears s_ah (each thread its own pixels)
                if (pend) ahstore_write<NPIX, NT, PPT>(a, pend_m, s_koff, s_cw, s_ah, tid);
                pend = false;
            }

            // P1: which pixels' rays enter which ellipsoids
            for (int e = 0; e < cnt; ++e) {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    bool hit = false;
                    if (alive[k]) {
                        ++n_cand;
                        hit = hit_test(sm + e * es, ck, ry[k]);
                    }
                    s_ah[e * NPIX + k * NT + tid] = 0.0f;
                    list_append(hit, (uint16_t)(k * NT + tid), &s_nh[e], s_hl + e * NPIX);
                }
            }
            __syncthreads();
            if (tid < 32) warp_prefix64(s_nh, cnt, s_ph);
            __syncthreads();

            if constexpr (NC > 0) {  // (without a colour network the phases are too short to cover it)
                const uint32_t c0n = c0 + CH;
                pre = c0n < rg.y;
                if (pre) {
                    if ((int)tid < min((int)(rg.y - c0n), CH))
                        cp_async4(s_gid + ((ci + 1) & 1) * (kMaxChunk / 2) + tid, a.vals + c0n + tid);
                    asm volatile("cp.async.commit_group;\n" ::: "memory");
                }
            }

            // P2: alpha_hat of every hit
            {
                const int nh = s_ph[cnt];
                int e = 0;
                for (int q = tid; q < nh; q += NT) {
                    while (q >= s_ph[e + 1]) ++e;
                    const int pix = s_hl[e * NPIX + (q - s_ph[e])];
                    const float *R = sm + e * es;
                    const PixRay r = load_ray(s_ray, pix);
                    Hit h;
                    float ah = 0.0f;
                    if (intersect(R, ck, r, h)) ah = integral<FORM>(R, R + kRecFloats, ns, ck, r, h);
                    s_ah[e * NPIX + pix] = ah;
                    ++n_hit;
                }
            }
            __syncthreads();

            // P3: compositing weights and termination, in list order
            uint64_t cmk[PPT];  // (alpha_hat store) entries of the chunk each pixel composited
#pragma unroll
            for (int k = 0; k < PPT; ++k) cmk[k] = 0ull;
            for (int e = 0; e < cnt; ++e) {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const int slot = k * NT + tid;
                    bool act = false;
                    float w = 0.0f;
                    if (alive[k]) {
                        const float ah = s_ah[e * NPIX + slot];
                        if (ah > 0.0f) {
                            ++n_comp;
                            w = T[k] * (1.0f - __expf(-ah));
                            tau[k] += ah;
                            T[k] = __expf(-tau[k]);
                            nwalk[k] = c0 - rg.x + e + 1;
                            act = true;
                            if constexpr (NC == 0) cmk[k] |= 1ull << e;
                            if constexpr (NC == 0) {
                                const float *R = sm + e * es;
                                C[k].x = fmaf(w, R[kRecRgb + 0], C[k].x);
                                C[k].y = fmaf(w, R[kRecRgb + 1], C[k].y);
                                C[k].z = fmaf(w, R[kRecRgb + 2], C[k].z);
                            }
                            if (T[k] < a.t_min) alive[k] = false;
                        }
                    }
                    // composited-pixel mask of this (tile, entry), one word per warp
                    const unsigned word = __ballot_sync(0xffffffffu, act);
                    if (lane_id() == 0 && a.cmask)
                        a.cmask[(int64_t)(c0 + e) * (NPIX / 32) + (slot >> 5)] = word;
                    if (NC > 0 || a.ahstore) {
                        if (lane_id() == 0) s_cw[e * (NPIX / 32) + (slot >> 5)] = word;
                    }
                    if constexpr (NC > 0) {
                        s_w[e * NPIX + slot] = act ? w : -1.0f;
                        list_append(act, (uint16_t)slot, &s_na[e], s_al + e * NPIX);
                    }
                }
            }

            if constexpr (NC > 0) {
                __syncthreads();
                if (tid < 32) warp_batch_prefix(s_na, cnt, 4, s_nb, s_pb);
                __syncthreads();
                // P4: colour of every composited pair, one warp per pass of 16 pairs of one entry
                const int np = s_pb[cnt];
                int e = 0;
                for (int q = tid >> 5; q < np; q += NT / 32) {
                    while (q >= s_pb[e + 1]) ++e;
                    warp_color_pass<NC, BF16>(sm + e * es + kRecFloats + den_stride(ns), s_ray, s_al + e * NPIX,
                                              (q - s_pb[e]) * 16, s_na[e], s_col + e * NPIX, 1, CH * NPIX);
                }
                if (tid < 32) {
                    // colour-store slice of the chunk (needed from P5 on; here it overlaps
                    // the other warps' colour passes)
                    if (a.colstore) store_slices(a, s_na, cnt, c0, s_pc, s_koff, s_cbase, s_blk_next, s_blk_end);
                }
                __syncthreads();
                // P5: accumulate in list order
                for (int e2 = 0; e2 < cnt; ++e2) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const int slot = k * NT + tid;
                        const float w = s_w[e2 * NPIX + slot];
                        if (w >= 0.0f) {
                            const float cx = s_col[(0 * CH + e2) * NPIX + slot], cy = s_col[(1 * CH + e2) * NPIX + slot],
                                        cz = s_col[(2 * CH + e2) * NPIX + slot];
                            C[k].x = fmaf(w, cx, C[k].x);
                            C[k].y = fmaf(w, cy, C[k].y);
                            C[k].z = fmaf(w, cz, C[k].z);
                            if (a.colstore) {
                                const uint32_t o = s_koff[e2];
                                if (o != kNoStore)
                                    a.colstore[o + mask_rank<NPIX>(s_cw + e2 * (NPIX / 32), slot)] =
                                        make_float4(cx, cy, cz, s_ah[e2 * NPIX + slot]);
                            }
                        }
                    }
                }
            }
            if constexpr (NC == 0) {
                // the alpha_hat store's writes of this chunk are made early in the next
                // chunk (or at the end of the tile), where barriers already are
                pend = a.ahstore != nullptr;
                pend_c0 = c0;
                pend_cnt = cnt;
#pragma unroll
                for (int k = 0; k < PPT; ++k) pend_m[k] = cmk[k];
            }
            bool any_alive = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) any_alive |= alive[k];
            if (__syncthreads_and(!any_alive)) break;
        }
        if constexpr (NC > 0) cp_async_wait_all();  // a copy for a chunk the early exit skipped must land first
        if constexpr (NC == 0) {
            if (pend) {  // the tile's last chunk
                __syncthreads();
                if (tid < 32) ahstore_slices<NPIX>(a, s_cw, pend_cnt, pend_c0, s_nb, s_pc, s_koff, s_cbase, s_blk_next,
                                             s_blk_end);
                __syncthreads();
                ahstore_write<NPIX, NT, PPT>(a, pend_m, s_koff, s_cw, s_ah, tid);
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            if (!inside[k]) continue;
            const int64_t p = V.pix_off + (int64_t)py[k] * V.width + px[k];
            a.image[3 * p + 0] = fmaf(T[k], a.bg[0], C[k].x);
            a.image[3 * p + 1] = fmaf(T[k], a.bg[1], C[k].y);
            a.image[3 * p + 2] = fmaf(T[k], a.bg[2], C[k].z);
            if (a.px_state) {
                a.px_state[p] = make_float4(C[k].x, C[k].y, C[k].z, tau[k]);
                a.px_nwalk[p] = nwalk[k];
            }
        }
        __syncthreads();
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

}  // namespace snp
