// snp_raster_bwd.cuh -- backward per-tile rasterizer.
//
// Persistent CTAs take tiles as in the forward and walk each tile's list in
// staged chunks.  Per chunk:
//   P1     each entry's pair list is its composited pixels in slot order, read
//          from the forward's composited masks (a pixel's position is its rank
//          among the mask's set bits);
//   P2/P4  alpha_hat and the colour of every composited pair are copied back from
//          the forward's colour store at that rank (without a colour network:
//          alpha_hat from the alpha_hat store, the colour from the staged record),
//          or -- where the store was full or is off -- recomputed;
//   P3/P5  each pixel replays its weights and the gradient of its colour with
//          respect to alpha_hat in list order;
//   P6     the per-pair gradients run as work items (colour passes first).
// The next chunk's record ids, store offsets and masks are copied in during P6,
// and the flush's bulk reductions read the accumulators while the next chunk
// starts.  With the forward's final colour C (no background) and optical depth
// tau_f:
//   C = sum_i c_i alpha_i T_i + T_f bg,  T_i = exp(-sum_{j<i} alpha_hat_j),
//   dC/dc_i = alpha_i T_i,
//   dC/dalpha_hat_i = T_{i+1} c_i - R_i - T_f bg,  R_i = sum_{j>i} c_j alpha_j T_j = C - prefix_i,
// which needs no division by (1 - alpha).  The chain rule then runs through the
// colour MLP, the closed-form integral (stable or literal Eq. 8) and the ray /
// ellipsoid geometry down to the projection record.  Per-pair gradients are
// reduced across each warp by a 32-value reduce-scatter, accumulated per list
// entry in shared memory across the warps, and added to the caller's gradient
// arrays with bulk asynchronous reductions, one per block per (tile, primitive).
#pragma once

#include "snp_raster.cuh"

namespace snp {

// Shared words for the composited masks of two backward chunks, the current one
// and the next one being copied in (chunk x tile pixels / 32 each; the backward
// chunk is at most 8 entries).
constexpr int kMaskWords = 512;

// Elements of one primitive's network record (snp_net_layout): every field
// 8-element aligned and padded.
__host__ __device__ constexpr int round8i(int x) { return (x + 7) & ~7; }
__host__ __device__ constexpr int net_stride(int ns, int nc, bool sh, bool dyn)
{
    return round8i(3 * ns) + 2 * round8i(ns) + 8 +
           (nc == 0 ? 0 : 8 + round8i(11 * nc) + round8i(nc) + round8i(nc * nc) + round8i(nc) + round8i(3 * nc) + 8) +
           (sh ? 48 : 0) + (dyn ? round8i(ns) + (sh ? 40 : 0) : 0);
}

// Per-entry gradient accumulator (floats):
//   [0, stride)             the primitive's network-gradient record in the caller's
//                           layout (snp_net_layout).  W1 and b1 hold gradients w.r.t.
//                           the staged rows w0 W1, w0 b1, and Wc2 is in mma fragment
//                           order (see warp_color_bwd_pass), until the flush;
//   [stride, +kGvFloats)    the per-(view, primitive) geometry gradient record;
//   [.., +n_c)              dL/dh0 (the folded first-layer bias).
// With the tensor-memory path (bwd_tmem) dL/dWc2 accumulates in TMEM, and the
// record has no Wc2 block: the fields after it, and the two blocks after the
// record, sit N_c^2 floats lower (the caller's layout has Wc2 followed only by
// bc2, Wc3 and bc3).  The flush adds the blocks to global memory with bulk
// asynchronous reductions (cp.reduce.async.bulk ... add.f32).
__host__ __device__ constexpr int acc_stride(int stride, int nc) { return stride + kGvFloats + nc; }

__device__ __forceinline__ void bulk_reduce_add(float *gdst, const float *ssrc, uint32_t bytes)
{
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;\n" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
}

// Flush the chunk's cnt entry accumulators: permute the Wc2 blocks to row-major
// and scale W1 / b1 by w0 in place (for a time-conditioned scene first setting
// dL/dW_t,k = xi dL/d(staged phase offset k), since the staged offset is
// w0 b1_k + xi W_t,k), then reduce every block into the caller's arrays with bulk
// asynchronous adds issued by thread 0.  Entries that no pixel composited (na[e]
// = 0: no work item touched their accumulators, which are still zero) are
// skipped.  All threads call it.  The reads of the bulk adds complete in the
// background: the kernel waits for them (thread 0) and clears the accumulators
// only in the next chunk, before its first accumulation.
// With TM, land holds the entries' dL/dWc2 blocks (row-major, N_c^2 floats each,
// written from tensor memory) and the accumulators are in the compact layout.
template <int NC, int NT, bool TM>
__device__ __forceinline__ void flush_chunk(const RasterArgs &a, float *acc, int vg, const uint32_t *s_gid, int cnt,
                                            const int *na, int64_t vn, int tid, int nt, float xi, const float *land)
{
    const int ns = a.n_sigma;
    if constexpr (NC > 0 && !TM) {  // (TM: the blocks came out of tensor memory row-major)
        // The fragment-order tiles (mn, nk) of row block mn hold exactly the rows
        // 16 mn .. 16 mn + 15 of Wc2, and in both layouts that block occupies the same
        // 16 NC words: one warp per entry permutes it block by block in place, through
        // registers.  Lane (g, t) takes the NC / 2 elements with its own (g, t) -- so
        // every read of the warp covers 32 banks -- in an order chosen so that the
        // writes do too: at step s it moves the element of tile nk = (g + s) mod 4
        // (+ 4 (s / 16) at N_c = 64) and fragment register i = 2 ((s / 8) mod 2) +
        // (g / 4 + s / 4) mod 2, whose row-major column 8 nk + 2 t + i mod 2 differs
        // across the 32 lanes.  No block barrier is needed.
        const int lane = tid & 31, g = lane >> 2, t = lane & 3;
        for (int e = tid >> 5; e < cnt; e += nt >> 5) {
            if (na[e] == 0) continue;  // uniform over the warp
            float *W = acc + e * vg + a.off_Wc2;
            for (int mn = 0; mn < NC / 16; ++mn) {
                float *B = W + mn * 16 * NC;
                float v[NC / 2];
#pragma unroll
                for (int s = 0; s < NC / 2; ++s) {
                    const int nk = ((g + s) & 3) | (NC == 64 ? ((s >> 4) & 1) << 2 : 0);
                    const int i = 2 * ((s >> 3) & 1) + (((g >> 2) + (s >> 2)) & 1);
                    v[s] = B[(nk * 4 + i) * 32 + lane];
                }
                __syncwarp();
#pragma unroll
                for (int s = 0; s < NC / 2; ++s) {
                    const int nk = ((g + s) & 3) | (NC == 64 ? ((s >> 4) & 1) << 2 : 0);
                    const int ih = (s >> 3) & 1, c = ((g >> 2) + (s >> 2)) & 1;
                    B[(g + 8 * ih) * NC + 8 * nk + 2 * t + c] = v[s];
                }
                __syncwarp();
            }
        }
    }
    if (NC == 0 && a.off_wt >= 0) {
        // same (entry, unit) -> thread map as the scaling loop below: no barrier needed
        for (int q = tid; q < cnt * (4 * ns); q += nt) {
            const int e = q / (4 * ns), r = q - e * (4 * ns);
            float *A = acc + e * vg;
            if (r >= 3 * ns && na[e] != 0) A[a.off_wt + r - 3 * ns] = xi * A[a.off_b1 + r - 3 * ns];
        }
    }
    for (int q = tid; q < cnt * (4 * ns); q += nt) {
        const int e = q / (4 * ns), r = q - e * (4 * ns);
        if (na[e] == 0) continue;
        float *A = acc + e * vg;
        if (r < 3 * ns) A[a.off_W1 + r] *= a.omega0;
        else A[a.off_b1 + (r - 3 * ns)] *= a.omega0;
    }
    // every thread's shared-memory writes become visible to the bulk copies' async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        constexpr int sw = TM ? NC * NC : 0;
        const int gvo = a.stride - sw;  // the geometry record's offset in the accumulator
        for (int e = 0; e < cnt; ++e) {
            if (na[e] == 0) continue;
            const int64_t gid = s_gid[e], prim = gid - vn;
            const float *A = acc + e * vg;
            if (a.g_net) {
                float *G = a.g_net + prim * a.stride;
                if constexpr (TM) {
                    const int w2 = a.off_Wc2, tail = a.stride - w2 - NC * NC;
                    bulk_reduce_add(G, A, (uint32_t)w2 * 4u);
                    bulk_reduce_add(G + w2, land + e * NC * NC, (uint32_t)(NC * NC) * 4u);
                    bulk_reduce_add(G + w2 + NC * NC, A + w2, (uint32_t)tail * 4u);
                } else {
                    bulk_reduce_add(G, A, (uint32_t)a.stride * 4u);
                }
            }
            bulk_reduce_add(a.g_view + gid * kGvFloats, A + gvo, kGvFloats * 4u);
            if constexpr (NC > 0) bulk_reduce_add(a.g_h0 + prim * NC, A + gvo + kGvFloats, NC * 4u);
        }
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    }
}

// N_sigma known at compile time (NS > 0): a pair's gradient values form one stream,
// the 5 NS density values (dL/dW1_k row, dL/db1_k, dL/dw2_k for k = 0 .. NS-1), then
// dL/db2, then the 22 slots of the geometry record, reduced across the warp 32 at a
// time as they are produced: ceil((5 NS + 23) / 32) reduce-scatters per batch (2 at
// N_sigma = 8, 6 at 32) instead of one per six density units plus one.  Put value
// idx of the stream into its group's slot; a full group (or the last) is reduced
// and each lane adds its sum to the accumulator A.  idx is a constant after
// unrolling, so v stays in registers.
template <int NS>
__device__ __forceinline__ void pack_put(float (&v)[32], int idx, float x, const RasterArgs &a, float *A, int gvo)
{
    constexpr int kTotal = 5 * NS + 23;
    v[idx & 31] = x;
    if ((idx & 31) == 31 || idx == kTotal - 1) {
#pragma unroll
        for (int i = (idx & 31) + 1; i < 32; ++i) v[i] = 0.0f;  // the tail of a last group
        const float r = warp_reduce_scatter32(v);
        const int q = (idx & ~31) + (int)lane_id();  // the stream index this lane summed
        if (r != 0.0f) {
            int dst = -1;
            if (q < 5 * NS) {
                const int k = q / 5, c = q - 5 * k;
                dst = c < 3 ? a.off_W1 + 3 * k + c : (c == 3 ? a.off_b1 + k : a.off_w2 + k);
            } else if (q == 5 * NS) {
                dst = a.off_b2;
            } else if (q < kTotal) {
                dst = gvo + (q - 5 * NS - 1);
            }
            if (dst >= 0) atomicAdd(A + dst, r);
        }
    }
}

// Density and geometry gradient of one (pixel, primitive) pair, reduced across
// the warp into the entry's shared-memory accumulator A (the colour MLP's part is
// a separate work item, warp_color_bwd_pass).  All 32 lanes call it together;
// lanes without a pair pass contrib = false (their contributions are zero).
// g_c: dL/dcolour, used for a constant colour only.
template <int NC, int FORM, int NS>
__device__ __forceinline__ void pair_backward(const RasterArgs &a, const float *R, const float *D, int ns,
                                              const CamK &ck,
                                              const PixRay &ry, bool contrib, float g_ah, float3 g_c, float *A,
                                              int gvo)
{
    const unsigned lane = lane_id();
    Hit h;
    if (!contrib || !intersect(R, ck, ry, h)) {
        // benign geometry for lanes that only take part in the warp reductions
        h.dx = h.dy = 0.0f;
        h.f = make_float3(0.f, 0.f, 0.f);
        h.dp = make_float3(1.f, 0.f, 0.f);
        h.w = make_float3(0.f, 0.f, 0.f);
        h.A = h.iA = h.h2 = 1.0f;
        h.W2 = h.fdp = h.s = h.t = 0.0f;
        h.half = 1.0f;
        g_ah = 0.0f;
        g_c = make_float3(0.f, 0.f, 0.f);
    }
    // ---- density (closed-form integral)
    const float inv_m = R[kRecInvM];
    const float mz = R[kRecMz], mz2 = R[kRecMz2];
    const float3 ac = make_float3(R[kRecAc + 0], R[kRecAc + 1], R[kRecAc + 2]);
    const float3 ocm = make_float3(R[kRecOcm + 0], R[kRecOcm + 1], R[kRecOcm + 2]);
    const float4 *W = reinterpret_cast<const float4 *>(D);
    const float *w2 = D + 4 * ns;
    const float b2 = w2[ns];
    const float3 dg = make_float3(fmaf(h.dx, ck.r0.x, h.dy * ck.r1.x), fmaf(h.dx, ck.r0.y, h.dy * ck.r1.y),
                                  fmaf(h.dx, ck.r0.z, h.dy * ck.r1.z));
    const float tm = h.t * inv_m, hm = h.half * inv_m;
    const float3 u = make_float3(fmaf(h.s, ac.x, tm * dg.x), fmaf(h.s, ac.y, tm * dg.y), fmaf(h.s, ac.z, tm * dg.z));
    const float gscale = g_ah * ry.gn;  // dL/dalpha_hat times |g|
    float3 g_u = make_float3(0.f, 0.f, 0.f), g_ocm = make_float3(0.f, 0.f, 0.f);
    float g_hm = 0.0f, S = b2, g_invm = 0.0f, g_t = 0.0f, g_half = 0.0f, g_b2;
    const float tin = h.t - h.half, tout = h.t + h.half;
    const float gS = gscale * 2.0f * h.half;
    float g_tout = 0.0f, g_tin = 0.0f;
    if constexpr (FORM == 0) {
        g_b2 = gS;
    } else {
        g_b2 = gscale * (tout - tin);
        g_tout = gscale * b2;
        g_tin = -gscale * b2;
    }
    // density unit k: its five gradient values (returned), and its share of the
    // sums the geometry part uses (accumulated)
    auto dens_k = [&](int k, float (&gw)[3], float &gb1, float &gw2) {
        const float4 w = W[k];
        const float wk = w2[k];
        const float g = fmaf(w.x, ry.g.x, fmaf(w.y, ry.g.y, w.z * ry.g.z));
        if constexpr (FORM == 0) {
            const float ph = fmaf(w.x, u.x, fmaf(w.y, u.y, fmaf(w.z, u.z, w.w)));
            const float th = g * hm;
            float sp, cp, st, ct;
            __sincosf(ph, &sp, &cp);
            __sincosf(th, &st, &ct);
            // sinc(th) and its derivative: series below |th| < kSincSeries, else one reciprocal
            const float t2 = th * th, rt = __fdividef(1.0f, th);
            const bool small = fabsf(th) < kSincSeries;
            const float sc = small ? sinc_series(t2) : st * rt;
            const float scp = small ? sinc_deriv_series(th, t2) : fmaf(th, ct, -st) * rt * rt;
            S = fmaf(wk * cp, sc, S);
            const float gphi = -gS * wk * sp * sc;
            const float gth = gS * wk * cp * scp;
            gw2 = gS * cp * sc;
            gw[0] = fmaf(gphi, u.x, gth * hm * ry.g.x);
            gw[1] = fmaf(gphi, u.y, gth * hm * ry.g.y);
            gw[2] = fmaf(gphi, u.z, gth * hm * ry.g.z);
            gb1 = gphi;
            g_u.x = fmaf(gphi, w.x, g_u.x);
            g_u.y = fmaf(gphi, w.y, g_u.y);
            g_u.z = fmaf(gphi, w.z, g_u.z);
            g_hm = fmaf(gth, g, g_hm);
        } else {
            const float ak = g * inv_m;
            const float psi = fmaf(w.x, ocm.x, fmaf(w.y, ocm.y, fmaf(w.z, ocm.z, w.w)));
            float s1, c1, s0, c0v;
            __sincosf(fmaf(ak, tout, psi), &s1, &c1);
            __sincosf(fmaf(ak, tin, psi), &s0, &c0v);
            const float ia = gscale != 0.0f ? __fdividef(1.0f, ak) : 0.0f;
            gw2 = gscale * (s1 - s0) * ia;
            const float gpsi = gscale * wk * (c1 - c0v) * ia;
            const float ga = gscale * wk * ((c1 * tout - c0v * tin) * ia - (s1 - s0) * ia * ia);
            gw[0] = fmaf(gpsi, ocm.x, ga * inv_m * ry.g.x);
            gw[1] = fmaf(gpsi, ocm.y, ga * inv_m * ry.g.y);
            gw[2] = fmaf(gpsi, ocm.z, ga * inv_m * ry.g.z);
            gb1 = gpsi;
            g_ocm.x = fmaf(gpsi, w.x, g_ocm.x);
            g_ocm.y = fmaf(gpsi, w.y, g_ocm.y);
            g_ocm.z = fmaf(gpsi, w.z, g_ocm.z);
            g_invm = fmaf(ga, g, g_invm);
            g_tout = fmaf(gscale * wk, c1, g_tout);
            g_tin = fmaf(-gscale * wk, c0v, g_tin);
        }
    };
    float pk[32];  // NS > 0: the current group of the packed gradient stream
    if constexpr (NS == 0) {
        for (int k0 = 0; k0 < ns; k0 += 6) {
            float vv[32];
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) {
                const int k = k0 + kk;
                float gw[3] = {0.f, 0.f, 0.f}, gb1 = 0.0f, gw2 = 0.0f;
                if (k < ns) dens_k(k, gw, gb1, gw2);
                vv[5 * kk + 0] = gw[0];
                vv[5 * kk + 1] = gw[1];
                vv[5 * kk + 2] = gw[2];
                vv[5 * kk + 3] = gb1;
                vv[5 * kk + 4] = gw2;
            }
            vv[30] = 0.0f;
            vv[31] = 0.0f;
            const float r = warp_reduce_scatter32(vv);
            const int kk = lane / 5, c = lane - 5 * kk, k = k0 + kk;
            if (lane < 30 && k < ns && r != 0.0f) {
                const int dst = c < 3 ? a.off_W1 + 3 * k + c : (c == 3 ? a.off_b1 + k : a.off_w2 + k);
                atomicAdd(A + dst, r);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            float gw[3] = {0.f, 0.f, 0.f}, gb1 = 0.0f, gw2 = 0.0f;
            dens_k(k, gw, gb1, gw2);
            pack_put<NS>(pk, 5 * k + 0, gw[0], a, A, gvo);
            pack_put<NS>(pk, 5 * k + 1, gw[1], a, A, gvo);
            pack_put<NS>(pk, 5 * k + 2, gw[2], a, A, gvo);
            pack_put<NS>(pk, 5 * k + 3, gb1, a, A, gvo);
            pack_put<NS>(pk, 5 * k + 4, gw2, a, A, gvo);
        }
        pack_put<NS>(pk, 5 * NS, g_b2, a, A, gvo);
    }
    // ---- geometry: (t, half) and u back to the record quantities
    float g_s = 0.0f;
    float3 g_ac = make_float3(0.f, 0.f, 0.f), g_dg = make_float3(0.f, 0.f, 0.f);
    if constexpr (FORM == 0) {
        // u = s ac + (t / m) dg; alpha_hat = 2 half |g| S; theta uses hm = half / m
        g_half = 2.0f * gscale * S + g_hm * inv_m;
        g_invm = g_hm * h.half + h.t * (g_u.x * dg.x + g_u.y * dg.y + g_u.z * dg.z);
        g_s = g_u.x * ac.x + g_u.y * ac.y + g_u.z * ac.z;
        g_t = inv_m * (g_u.x * dg.x + g_u.y * dg.y + g_u.z * dg.z);
        g_ac = make_float3(h.s * g_u.x, h.s * g_u.y, h.s * g_u.z);
        g_dg = make_float3(tm * g_u.x, tm * g_u.y, tm * g_u.z);
    } else {
        g_t = g_tout + g_tin;
        g_half = g_tout - g_tin;
    }
    // t = mz + s, s = -mz (f . dp) / A, half = sqrt(h2 / A), h2 = 1 - mz^2 |w|^2 / A
    const float g_st = g_s + g_t;
    float g_mz = g_t - g_st * h.fdp * h.iA;
    const float g_fdp = -mz * h.iA * g_st;
    float g_iA = -mz * h.fdp * g_st;
    const float gx = __fdividef(g_half, 2.0f * h.half);
    const float g_h2 = gx * h.iA;
    g_iA += gx * h.h2;
    g_mz += 2.0f * mz * (-g_h2 * h.W2 * h.iA);
    const float g_W2 = -g_h2 * mz2 * h.iA;
    g_iA += -g_h2 * mz2 * h.W2;
    const float3 g_w = make_float3(2.0f * g_W2 * h.w.x, 2.0f * g_W2 * h.w.y, 2.0f * g_W2 * h.w.z);
    const float g_A = -g_iA * h.iA * h.iA;
    const float3 e = make_float3(R[kRecE + 0], R[kRecE + 1], R[kRecE + 2]);
    // dp = e + f:  dL/ddp from A = dp.dp and from fdp = f.dp
    const float3 g_dp = make_float3(fmaf(2.0f * g_A, h.dp.x, g_fdp * h.f.x), fmaf(2.0f * g_A, h.dp.y, g_fdp * h.f.y),
                                    fmaf(2.0f * g_A, h.dp.z, g_fdp * h.f.z));
    // w = e x f:  dL/de = f x g_w,  dL/df = g_w x e
    float3 g_e = make_float3(h.f.y * g_w.z - h.f.z * g_w.y + g_dp.x, h.f.z * g_w.x - h.f.x * g_w.z + g_dp.y,
                             h.f.x * g_w.y - h.f.y * g_w.x + g_dp.z);
    const float3 g_f = make_float3(g_w.y * e.z - g_w.z * e.y + g_dp.x + g_fdp * h.dp.x,
                                   g_w.z * e.x - g_w.x * e.z + g_dp.y + g_fdp * h.dp.y,
                                   g_w.x * e.y - g_w.y * e.x + g_dp.z + g_fdp * h.dp.z);
    // f = G[:,0] dx + G[:,1] dy;  dg = dx r0 + dy r1;  dx = (px + .5 - U_c) / fx
    const float g_dx = g_f.x * R[kRecG + 0] + g_f.y * R[kRecG + 3] + g_f.z * R[kRecG + 6] +
                       g_dg.x * ck.r0.x + g_dg.y * ck.r0.y + g_dg.z * ck.r0.z;
    const float g_dy = g_f.x * R[kRecG + 1] + g_f.y * R[kRecG + 4] + g_f.z * R[kRecG + 7] +
                       g_dg.x * ck.r1.x + g_dg.y * ck.r1.y + g_dg.z * ck.r1.z;

    float gv[22];  // the geometry record's slots 0 .. 21 (22, 23 stay zero)
    gv[kGvG + 0] = g_f.x * h.dx; gv[kGvG + 1] = g_f.x * h.dy;
    gv[kGvG + 2] = g_f.y * h.dx; gv[kGvG + 3] = g_f.y * h.dy;
    gv[kGvG + 4] = g_f.z * h.dx; gv[kGvG + 5] = g_f.z * h.dy;
    gv[kGvE + 0] = g_e.x; gv[kGvE + 1] = g_e.y; gv[kGvE + 2] = g_e.z;
    gv[kGvMz] = g_mz;
    gv[kGvU] = -g_dx * ck.ifx;
    gv[kGvV] = -g_dy * ck.ify;
    gv[kGvAc + 0] = g_ac.x; gv[kGvAc + 1] = g_ac.y; gv[kGvAc + 2] = g_ac.z;
    gv[kGvInvM] = g_invm;
    gv[kGvOcm + 0] = g_ocm.x; gv[kGvOcm + 1] = g_ocm.y; gv[kGvOcm + 2] = g_ocm.z;
    gv[kGvRgb + 0] = NC == 0 ? g_c.x : 0.0f;
    gv[kGvRgb + 1] = NC == 0 ? g_c.y : 0.0f;
    gv[kGvRgb + 2] = NC == 0 ? g_c.z : 0.0f;
    if constexpr (NS == 0) {
        float vv[32];
#pragma unroll
        for (int q = 0; q < 22; ++q) vv[q] = gv[q];
        vv[22] = 0.0f;
        vv[23] = 0.0f;
        vv[24] = g_b2;
#pragma unroll
        for (int q = 25; q < 32; ++q) vv[q] = 0.0f;
        const float r = warp_reduce_scatter32(vv);
        if (r != 0.0f) {
            if (lane < (unsigned)kGvFloats) atomicAdd(A + gvo + lane, r);
            else if (lane == 24) atomicAdd(A + a.off_b2, r);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 22; ++q) pack_put<NS>(pk, 5 * NS + 1 + q, gv[q], a, A, gvo);
    }

}

// Whether the backward accumulates dL/dWc2 in tensor memory (tcgen05; N_c = 64 on
// 256-thread tiles) instead of shared-memory atomics.  The N_c = 32 form below
// (warp_color_bwd_pass) is built and correct but measured slower than the atomics
// there: its operand tiles cost a chunk entry at two CTAs per SM, and the short
// passes leave the per-pass MMA issue exposed.
__host__ __device__ constexpr bool bwd_tmem(int ts, int nc) { return nc == 64 && ts >= 16; }
// Per-warp operand tiles of the tensor-memory path (bytes).  N_c = 64: A hi, A lo,
// B hi, B lo, each 64 x 16 bf16.  N_c = 32: A = the hi and lo halves of dL/da2^T
// stacked into one 64 x 16 tile, B hi, B lo (32 x 16 each).
__host__ __device__ constexpr int tmem_stage_bytes(int nc) { return nc == 64 ? 8192 : 4096; }
// With the tensor-memory path the per-entry accumulator has no Wc2 block (the
// record's fields after it move down by N_c^2 floats): at the chunk's end the
// accumulators leave tensor memory into the warps' operand tiles, which are free
// then, one N_c x N_c block per entry.  So a chunk holds at most this many entries.
__host__ __device__ constexpr int tmem_max_chunk(int nt, int nc)
{
    return (nt / 32) * tmem_stage_bytes(nc) / (nc * nc * 4);
}
__host__ __device__ constexpr int tmem_wc2_floats(int ts, int nc) { return bwd_tmem(ts, nc) ? nc * nc : 0; }

template <int TS>
__host__ __device__ inline size_t bwd_smem_bytes(int nc, int ns, int chunk, int stride)
{
    constexpr int NPIX = TileCfg<TS>::NPIX;
    const size_t per_entry = (size_t)(entry_stride(ns, nc) + acc_stride(stride, nc) - tmem_wc2_floats(TS, nc)) * 4 +
                             (size_t)NPIX * (5 * 4 + 2);
    const size_t stage = bwd_tmem(TS, nc) ? (size_t)(TileCfg<TS>::NT / 32) * tmem_stage_bytes(nc) + 128 : 0;
    return NPIX * (32 + 12) + (size_t)chunk * per_entry + stage;
}

// NS > 0: built for n_sigma = NS (the density loop unrolled, its gradients packed;
// see pack_put); NS = 0: any n_sigma.
template <int TS, int NC, int FORM, bool BF16, int NS>
__global__ void __launch_bounds__(TileCfg<TS>::NT, bwd_min_blocks(TS, NC)) k_raster_bwd(RasterArgs a)
{
    constexpr int NT = TileCfg<TS>::NT;
    constexpr int NPIX = TileCfg<TS>::NPIX;
    constexpr int PPT = TileCfg<TS>::PPT;
    extern __shared__ float4 smem4[];
    const int CH = a.chunk;
    const int ns = NS > 0 ? NS : a.n_sigma;
    const int es = entry_stride(ns, NC);
    constexpr int SW = tmem_wc2_floats(TS, NC);  // Wc2 floats not in the accumulator (TMEM path)
    const int vg = acc_stride(a.stride, NC) - SW;
    const int gvo = a.stride - SW;  // offset of the geometry record in an accumulator
    float4 *s_ray = smem4;                                 // [2 NPIX] pixel rays
    float *s_dl = reinterpret_cast<float *>(smem4 + 2 * NPIX);  // [3][NPIX] dL/dC of the tile's pixels
    float *sm = s_dl + 3 * NPIX;                           // [CH][es] staged entries
    float *acc = sm + CH * es;                             // [CH][vg] per-entry gradient sums
    // [CH][NPIX] per composited pair: colour (x, y, z) and alpha_hat (w), which P3/P5
    // replace by dL/dalpha_hat (the layout of a colour-store record)
    float4 *s_cs = reinterpret_cast<float4 *>(acc + CH * vg);
    float *s_w = reinterpret_cast<float *>(s_cs + CH * NPIX);  // [CH][NPIX] weights of the composited pairs
    uint16_t *s_al = reinterpret_cast<uint16_t *>(s_w + CH * NPIX);  // [CH][NPIX] pair lists
    constexpr bool TM = bwd_tmem(TS, NC);
    constexpr bool kEarly = NC == 0 || TM;  // begin the next chunk before the flush (below)
    // TM: per warp, the operand tiles of its tcgen05.mma (128-byte aligned)
    char *s_stage = reinterpret_cast<char *>(
        (reinterpret_cast<uintptr_t>(s_al + CH * NPIX) + 127) & ~static_cast<uintptr_t>(127));
    __shared__ uint32_t s_gid[kMaxChunk];
    __shared__ uint32_t s_koff[64];         // colour-store offsets of the chunk's keys (two halves)
    __shared__ bool s_stored;               // every composited pair of the chunk is in the store
    __shared__ uint32_t s_cmw[kMaskWords];  // composited-mask words of the chunk (two halves)
    // s_na: composited pairs per entry of the current and the next chunk (two halves)
    __shared__ int s_na[66], s_pa[65], s_nb[65], s_pb[65], s_np[65], s_pp[65];
    __shared__ int s_view, s_item;
    __shared__ int s_item6;  // P6 item counter (items past the first one of each warp)
    __shared__ uint32_t s_maxwalk;
    // TM: per-warp MMA barriers, the TMEM base address, the issue lock and per-entry
    // "accumulator written in this chunk" flags
    __shared__ __align__(8) uint64_t s_tmbar[NT / 32];
    __shared__ uint32_t s_tmaddr;
    __shared__ int s_tmlock;
    __shared__ int s_tmstart[kMaxChunk / 2];

    const int tid = threadIdx.x;
    const unsigned lane = lane_id();
    const int wid = tid >> 5;
    // the forward's per-pair store: (colour, alpha_hat) with a colour network, else alpha_hat
    const bool has_store = NC > 0 ? a.colstore != nullptr : a.ahstore != nullptr;
    for (int q = tid; q < CH * vg; q += NT) acc[q] = 0.0f;
    // TM: TMEM columns for the chunk's accumulators (entry e at columns N_c e; 64
    // lanes by N_c columns at N_c = 64, 64 lanes by 32 columns at N_c = 32, where
    // the hi and lo halves of dL/da2 are stacked along M)
    uint32_t tm_cols = 32;
    while ((int)tm_cols < (NC > 0 ? NC : 1) * CH) tm_cols <<= 1;
    int ncommit = 0;
    if constexpr (TM) {
        if (tid < NT / 32) mbar_init(&s_tmbar[tid], 1);
        if (tid == 0) {
            s_tmlock = 0;
            mbar_init_fence();
        }
        if (wid == 0) tmem_alloc(&s_tmaddr, tm_cols);
        tc_fence_before_sync();
        __syncthreads();
        tc_fence_after_sync();
        // test hook: phase 0 of this barrier completes only after this warp's first MMA
        // group, which has not been issued yet, so this wait runs out
        if (a.test_stuck_wait && tid == 0 && !mbar_wait_bounded(&s_tmbar[0], 0u, 1 << 12)) *a.wait_status = 1;
    }
    int clear_n = 0;  // float4s of accumulators the next chunk clears (after the bulk reads)

    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(a.work_counter, 1);
            s_maxwalk = 0;
        }
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
        PixRay ry[PPT];
        float3 Cf[PPT], dL[PPT], pref[PPT];
        float tau[PPT], bgdot[PPT];
        uint32_t nwalk[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            int lx, ly;
            tile_pixel<TS>(tid, k, lx, ly);
            const int px = tx * TS + lx, py = ty * TS + ly;
            const bool inside = px < V.width && py < V.height;
            ry[k] = pixel_ray(V, px, py);
            store_ray(s_ray, k * NT + tid, ry[k]);
            Cf[k] = make_float3(0.f, 0.f, 0.f);
            dL[k] = make_float3(0.f, 0.f, 0.f);
            pref[k] = make_float3(0.f, 0.f, 0.f);
            float tau_f = 0.0f;
            nwalk[k] = 0;
            if (inside) {
                const int64_t p = V.pix_off + (int64_t)py * V.width + px;
                const float4 s4 = a.px_state[p];
                Cf[k] = make_float3(s4.x, s4.y, s4.z);
                tau_f = s4.w;
                nwalk[k] = a.px_nwalk[p];
                dL[k] = make_float3(a.dL_dimage[3 * p + 0], a.dL_dimage[3 * p + 1], a.dL_dimage[3 * p + 2]);
                atomicMax(&s_maxwalk, nwalk[k]);
            }
            bgdot[k] = __expf(-tau_f) * (dL[k].x * a.bg[0] + dL[k].y * a.bg[1] + dL[k].z * a.bg[2]);
            tau[k] = 0.0f;
            s_dl[k * NT + tid] = dL[k].x;
            s_dl[NPIX + k * NT + tid] = dL[k].y;
            s_dl[2 * NPIX + k * NT + tid] = dL[k].z;
        }
        const uint2 rg = a.ranges[tile];
        const int64_t vn = (int64_t)v * a.n;
        __syncthreads();
        const uint32_t maxwalk = s_maxwalk;

        // Per chunk: its keys' record ids, colour-store offsets, composited masks and
        // composited counts, in one of two halves of s_gid / s_koff / s_cmw / s_na; the
        // next chunk's ids, offsets and masks are copied into the other half (4-byte
        // cp.async) while this chunk runs P6.  Before this chunk's flush the next chunk's
        // staging copies are issued, and with kEarly P1 also builds its pair lists and
        // issues its store copies there, so that the copies land while the flush runs.
        // (Measured: without a colour network 37.1 -> 35.7 ms on the 8-view 800 x 800
        // speed protocol.  At N_c = 32, two CTAs per SM, P1 before the flush was 0.6 ms
        // slower, the staging copies alone there 0.3 ms faster: that kernel builds its
        // lists after the flush.)
        uint32_t cm[PPT];  // per pixel: entries of the chunk whose lists were built last
        // Chunk (c0b, cib): its ids, offsets and masks (copied in during the previous
        // chunk's P6 if `prefetched`, else loaded here) and its staging copies.
        auto stage_begin = [&](uint32_t c0b, int cib, bool prefetched) {
            const int cntb = min((int)(rg.y - c0b), CH);
            uint32_t *const bg = s_gid + (cib & 1) * (kMaxChunk / 2);
            uint32_t *const bko = s_koff + (cib & 1) * 32;
            uint32_t *const bmw = s_cmw + (cib & 1) * (kMaskWords / 2);
            int *const bna = s_na + (cib & 1) * 33;
            if (prefetched) {
                cp_async_wait_all();
            } else {
                if (tid < cntb) {
                    bg[tid] = a.vals[c0b + tid];
                    bko[tid] = has_store ? a.key_off[c0b + tid] : kNoStore;
                }
                // composited masks of the chunk's entries (none past the tile's walk length)
                for (int i = tid; i < cntb * (NPIX / 32); i += NT) {
                    const int e = i / (NPIX / 32);
                    bmw[i] = c0b - rg.x + e < maxwalk ? a.cmask[(int64_t)c0b * (NPIX / 32) + i] : 0u;
                }
            }
            if constexpr (TM) {
                if (tid < cntb) s_tmstart[tid] = 0;
            }
            __syncthreads();
            // staging copies in flight through P1, which needs only the masks; one wait
            // covers them and P1's store copies
            if constexpr (NC > 0) stage_chunk_issue<NC, BF16>(sm, bg, cntb, vn, a, es);
            else stage_issue_flat(sm, bg, cntb, vn, a, es);
        };
        // P1 of chunk (c0b, cib), whose ids, offsets and masks are in place
        auto build_lists = [&](uint32_t c0b, int cib) {
            const int cntb = min((int)(rg.y - c0b), CH);
            const uint32_t *const bko = s_koff + (cib & 1) * 32;
            const uint32_t *const bmw = s_cmw + (cib & 1) * (kMaskWords / 2);
            int *const bna = s_na + (cib & 1) * 33;
            // P1: the pixels that composited each entry, from the forward's masks (entries
            // at or past the tile's walk length were composited by no pixel)
#pragma unroll
            for (int k = 0; k < PPT; ++k) cm[k] = 0u;
            // Each entry's pair list is its composited pixels in slot order: a pixel's
            // position is its rank among the set bits of the entry's mask (no atomics).
            for (int e = 0; e < cntb; ++e) {
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const int slot = k * NT + tid;
                    const unsigned word = bmw[e * (NPIX / 32) + (slot >> 5)];
                    const bool act = (word >> lane) & 1u;
                    cm[k] |= (uint32_t)act << e;
                    if (act) {
                        const uint32_t rank = mask_rank<NPIX>(bmw + e * (NPIX / 32), slot);
                        s_al[e * NPIX + rank] = (uint16_t)slot;
                        const uint32_t o = bko[e];
                        if (o != kNoStore) {
                            if constexpr (NC > 0) {
                                // the pair's (colour, alpha_hat) from the forward's store
                                cp_async16(s_cs + e * NPIX + slot, a.colstore + o + rank);
                            } else {
                                // alpha_hat from the store (the colour is the staged record's)
                                cp_async4(reinterpret_cast<float *>(s_cs + e * NPIX + slot) + 3, a.ahstore + o + rank);
                            }
                        }
                    }
                }
            }
            if (tid < cntb) {
                int c = 0;
                for (int w = 0; w < NPIX / 32; ++w) c += __popc(bmw[tid * (NPIX / 32) + w]);
                bna[tid] = c;
            }
        };

        bool pre = false;
        int ci = 0;
        for (uint32_t c0 = rg.x; c0 < rg.y && c0 - rg.x < maxwalk; c0 += CH, ++ci) {
            const int cnt = min((int)(rg.y - c0), CH);
            uint32_t *const cg = s_gid + (ci & 1) * (kMaxChunk / 2);
            uint32_t *const cko = s_koff + (ci & 1) * 32;
            const int *const na = s_na + (ci & 1) * 33;
            // A chunk after the first had its staging copies issued before the previous
            // chunk's flush, and with kEarly its pair lists built there too.
            if (ci == 0) stage_begin(c0, 0, false);
            if (ci == 0 || !kEarly) build_lists(c0, ci);
            if (tid == 0) s_item6 = 0;
            cp_async_wait_all();  // this chunk's staging and store copies
            if constexpr (NC == 0) stage_shift_flat<BF16>(sm, cg, cnt, vn, a, es, V.time);
            // the previous chunk's bulk adds have read its accumulators by now
            if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
            __syncthreads();
            {
                float4 *A4 = reinterpret_cast<float4 *>(acc);
                for (int q = tid; q < clear_n; q += NT) A4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (tid < 32) {
                warp_prefix64(na, cnt, s_pa);
                warp_batch_prefix(na, cnt, 5, s_nb, s_pb);  // density items: 32 pairs
                warp_batch_prefix(na, cnt, 4, s_np, s_pp);  // colour items: 16 pairs
                const bool miss = (int)lane < cnt && na[lane] > 0 && cko[lane] == kNoStore;
                const bool any = __any_sync(0xffffffffu, miss);
                if (lane == 0) s_stored = !any;
            }
            __syncthreads();
            const bool stored = s_stored;
            // P2: alpha_hat of every composited pair (per thread), then P4: their colours
            // (per warp, 16 pairs of one entry); independent, so one phase.  With the
            // store both come from the forward (without a colour network the colour is
            // the staged record's).
            {
                const int np2 = s_pa[cnt];
                int e = 0;
                for (int q = tid; q < (stored ? 0 : np2); q += NT) {
                    while (q >= s_pa[e + 1]) ++e;
                    const int pix = s_al[e * NPIX + (q - s_pa[e])];
                    const float *R = sm + e * es;
                    const PixRay r = load_ray(s_ray, pix);
                    Hit h;
                    float ah = 0.0f;
                    if (intersect(R, ck, r, h)) ah = integral<FORM>(R, R + kRecFloats, ns, ck, r, h);
                    s_cs[e * NPIX + pix].w = ah;
                }
            }
            if constexpr (NC > 0) {
                if (!stored) {
                    const int np = s_pp[cnt];
                    int e = 0;
                    for (int q = wid; q < np; q += NT / 32) {
                        while (q >= s_pp[e + 1]) ++e;
                        warp_color_pass<NC, BF16>(sm + e * es + kRecFloats + den_stride(ns), s_ray,
                                                  s_al + e * NPIX, (q - s_pp[e]) * 16, na[e],
                                                  reinterpret_cast<float *>(s_cs + e * NPIX), 4, 1);
                    }
                }
            }
            __syncthreads();
            // P3/P5 (per pixel, over its composited entries in list order): the weights
            // w_i = T_i (1 - e^{-alpha_hat_i}) and
            // dL/dalpha_hat_i = dL . (T_{i+1} c_i - (C - prefix_i)) - T_f dL . bg
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int slot = k * NT + tid;
                for (uint32_t m = cm[k]; m != 0u; m &= m - 1u) {
                    const int e = __ffs(m) - 1;
                    const float4 cs = s_cs[e * NPIX + slot];
                    const float ah = cs.w;
                    const float w = __expf(-tau[k]) * (1.0f - __expf(-ah));
                    tau[k] += ah;
                    const float Tn = __expf(-tau[k]);
                    s_w[e * NPIX + slot] = w;
                    float3 col;
                    if constexpr (NC > 0) {
                        col = make_float3(cs.x, cs.y, cs.z);
                    } else {
                        const float *R = sm + e * es;
                        col = make_float3(R[kRecRgb + 0], R[kRecRgb + 1], R[kRecRgb + 2]);
                    }
                    pref[k].x = fmaf(w, col.x, pref[k].x);
                    pref[k].y = fmaf(w, col.y, pref[k].y);
                    pref[k].z = fmaf(w, col.z, pref[k].z);
                    s_cs[e * NPIX + slot].w = dL[k].x * (Tn * col.x - (Cf[k].x - pref[k].x)) +
                                              dL[k].y * (Tn * col.y - (Cf[k].y - pref[k].y)) +
                                              dL[k].z * (Tn * col.z - (Cf[k].z - pref[k].z)) - bgdot[k];
                }
            }
            __syncthreads();
            // the next chunk's ids, store offsets and masks, in flight through P6
            const uint32_t c0n = c0 + CH;
            pre = c0n < rg.y && c0n - rg.x < maxwalk;
            if (pre) {
                const int cntn = min((int)(rg.y - c0n), CH);
                uint32_t *const ng = s_gid + ((ci + 1) & 1) * (kMaxChunk / 2);
                uint32_t *const nko = s_koff + ((ci + 1) & 1) * 32;
                uint32_t *const nmw = s_cmw + ((ci + 1) & 1) * (kMaskWords / 2);
                if (tid < cntn) {
                    cp_async4(ng + tid, a.vals + c0n + tid);
                    if (has_store) cp_async4(nko + tid, a.key_off + c0n + tid);
                    else nko[tid] = kNoStore;
                }
                for (int i = tid; i < cntn * (NPIX / 32); i += NT) {
                    const int e = i / (NPIX / 32);
                    if (c0n - rg.x + e < maxwalk) cp_async4(nmw + i, a.cmask + (int64_t)c0n * (NPIX / 32) + i);
                    else nmw[i] = 0u;
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            // P6: per-pair gradients.  Work items: colour-MLP passes of 16 pairs of one
            // entry (tensor cores), then density / geometry batches of 32 pairs of one
            // entry (per-lane chain, warp reductions).  The costlier colour passes go
            // first and warps take the next item from a shared counter as they finish,
            // so the phase ends on short items.
            {
                const int nb = s_pb[cnt], np = NC > 0 ? s_pp[cnt] : 0;
                int e = 0, ec = 0;
                int it = wid;
                while (it < nb + np) {
                    if (NC > 0 && it < np) {
                        if constexpr (NC > 0) {
                            while (it >= s_pp[ec + 1]) ++ec;
                            float *A = acc + ec * vg;
                            TmemPass tp{};
                            if constexpr (TM) {
                                tp.stage_ptr = s_stage + wid * tmem_stage_bytes(NC);
                                tp.stage = cvta_smem(tp.stage_ptr);
                                tp.bar = &s_tmbar[wid];
                                tp.d_tmem = s_tmaddr + (uint32_t)NC * (uint32_t)ec;
                                tp.started = &s_tmstart[ec];
                                tp.lock = &s_tmlock;
                                tp.wait_status = a.wait_status;
                            }
                            warp_color_bwd_pass<NC, BF16, TM>(sm + ec * es + kRecFloats + den_stride(ns), s_ray,
                                                              s_al + ec * NPIX, (it - s_pp[ec]) * 16, na[ec],
                                                              s_w + ec * NPIX, s_dl, NPIX,
                                                              reinterpret_cast<const float *>(s_cs + ec * NPIX), 4,
                                                              1, A + a.off_Wc1, A + gvo + kGvFloats,
                                                              A + a.off_Wc2, A + a.off_Wc3 - SW,
                                                              A + a.off_bc2 - SW, A + a.off_bc3 - SW, tp, ncommit);
                        }
                    } else {
                        const int q = it - np;
                        while (q >= s_pb[e + 1]) ++e;
                        const int kk = (q - s_pb[e]) * 32 + (int)lane;
                        const bool valid = kk < na[e];
                        const int pix = valid ? s_al[e * NPIX + kk] : 0;
                        const PixRay r = load_ray(s_ray, pix);
                        const float *R = sm + e * es;
                        float3 g_c = make_float3(0.f, 0.f, 0.f);
                        if constexpr (NC == 0) {
                            // dL/dc_i = w_i dL
                            const float wi = valid ? s_w[e * NPIX + pix] : 0.0f;
                            g_c = make_float3(wi * s_dl[pix], wi * s_dl[NPIX + pix], wi * s_dl[2 * NPIX + pix]);
                        }
                        pair_backward<NC, FORM, NS>(a, R, R + kRecFloats, ns, ck, r, valid, s_cs[e * NPIX + pix].w, g_c,
                                                acc + e * vg, gvo);
                    }
                    int nx = 0;
                    if (lane == 0) nx = atomicAdd(&s_item6, 1) + NT / 32;
                    it = __shfl_sync(0xffffffffu, nx, 0);
                }
            }
            if constexpr (TM) {
                // this warp's last MMAs have completed (and read its operand tiles)
                if (ncommit > 0 && !mbar_wait_bounded(&s_tmbar[wid], (uint32_t)((ncommit - 1) & 1)))
                    *a.wait_status = 1;
                tc_fence_before_sync();
            }
            __syncthreads();
            float *land = reinterpret_cast<float *>(s_stage);  // TM: entry e's dL/dWc2 at e N_c^2
            if constexpr (TM) {
                // dL/dWc2 of every composited entry from TMEM into the (now idle) operand
                // tiles, row-major.  The M = 64 accumulator keeps rows 16 j .. 16 j + 15 in
                // TMEM lanes 32 j .. 32 j + 15, which only warps w with w % 4 = j can read.
                tc_fence_after_sync();
                const int q = wid & 3;
                if constexpr (NC == 64) {
                    // warp w: rows 16 (w % 4) .. + 15, columns 32 (w / 4) .. + 31
                    const int half = wid >> 2;
                    for (int e = 0; e < cnt; ++e) {
                        if (na[e] == 0) continue;
                        uint32_t r[32];
                        tmem_ld32(s_tmaddr + ((uint32_t)(32 * q) << 16) + 64u * (uint32_t)e + 32u * (uint32_t)half, r);
                        if (lane < 16) {
                            // The 16 rows are 256 bytes apart, so stores of the same 16-byte piece
                            // of every row hit the same four banks (16-way).  Lane l rotates its
                            // eight pieces by rot = l % 8 (a barrel shift of static register
                            // indices): store j then writes piece (j + rot) % 8, and the 16 lanes
                            // of one store cover all 32 banks.
                            const int rot = (int)lane & 7;
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                const bool b = (rot >> k) & 1;
                                uint32_t t[32];
#pragma unroll
                                for (int i = 0; i < 32; ++i) t[i] = b ? r[(i + (4 << k)) & 31] : r[i];
#pragma unroll
                                for (int i = 0; i < 32; ++i) r[i] = t[i];
                            }
                            float4 *dst = reinterpret_cast<float4 *>(land + e * NC * NC + (16 * q + (int)lane) * 64 +
                                                                     32 * half);
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                dst[(j + rot) & 7] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                                                 __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                        }
                    }
                } else {
                    // N_c = 32: lane l < 8 of warp w holds output unit 8 (w % 4) + l from the
                    // hi half of dL/da2, lane l + 8 the same unit from the lo half; their sum
                    // is the row.  Warps w and w + 4 take alternate entries.
                    for (int e = wid >> 2; e < cnt; e += 2) {
                        if (na[e] == 0) continue;
                        uint32_t r[32];
                        tmem_ld32(s_tmaddr + ((uint32_t)(32 * q) << 16) + 32u * (uint32_t)e, r);
                        float v[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            v[j] = __uint_as_float(r[j]);
                            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 8);
                        }
                        if (lane < 8) {
                            float4 *dst = reinterpret_cast<float4 *>(land + e * NC * NC + (8 * q + (int)lane) * 32);
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        }
                    }
                }
                tc_fence_before_sync();
                __syncthreads();
            }
            // the next chunk's staging copies (and with kEarly its lists) before this
            // chunk's flush, so that the copies land meanwhile
            if (pre) {
                stage_begin(c0n, ci + 1, true);
                if constexpr (kEarly) build_lists(c0n, ci + 1);
            }
            flush_chunk<NC, NT, TM>(a, acc, vg, cg, cnt, na, vn, tid, NT, V.time, land);
            clear_n = cnt * vg / 4;
        }
        __syncthreads();
    }
    // the bulk reductions must complete before the CTA exits
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    if constexpr (TM) {
        // every MMA completed at its chunk's end; give the columns back
        tc_fence_before_sync();
        __syncthreads();
        tc_fence_after_sync();
        if (wid == 0) tmem_dealloc(s_tmaddr, tm_cols);
    }
}

}  // namespace snp
