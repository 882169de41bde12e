// Top-K forward render (included by one translation unit per feature type,
// so that the two sets of template instances compile in parallel).
//
// Front-to-back alpha compositing of the depth-sorted tile lists (Sec. 3.1,
// Eq. 2) with Top-K Hard Selection before the C-channel feature
// accumulation (Sec. 3.4, Eq. 7).  One CTA renders one TS x TS tile, one
// thread per pixel.
// Phase 1: batches of BATCH surfel records are staged in shared memory by the
//   CTA; every thread intersects its pixel ray with each staged surfel,
//   composites colour and transmittance and keeps its K largest blending
//   weights in registers (ties keep the earlier surfel).  A warp leaves the
//   batch loop as soon as all its pixels have stopped; the CTA stops staging
//   once every pixel has.
// Phase 2: the CTA gathers only the K selected feature rows per pixel
//   (16-byte loads: 8 bf16 or 4 f32 channels), weights them in FP32 and writes
//   channel-last output with consecutive lanes on consecutive 16-byte chunks.
// Variants: FRONT takes the first K contributors instead of the K largest
// weights; AUX also accumulates the sensor outputs (expected and median
// depth, facing normal) over every contributor and applies the low-pass
// filter when the parameters ask for it; LOSS evaluates the training loss
// (L2 on the features, L1 on the colour) and its gradients where F and rgb
// are formed; SORT (with LOSS) first depth-sorts the CTA's own tile list
// (sort_tile), so that no sort kernel runs before it.
//
// The accumulation is a sparse gather-weighted sum, not a dense contraction,
// so no tensor cores are involved.
#pragma once

#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"
#include "sort.cuh"

#include <algorithm>
#include <climits>

namespace fss {

namespace topk_detail {

__device__ __forceinline__ int next_tile(const Cams& cams, const FwdArgs& a, int* s_tile, bool first) {
    return next_tile_q(a.persistent, &a.st->work, s_tile, first, cams);
}

}  // namespace topk_detail

using topk_detail::next_tile;

// ---------------------------------------------------------------------------
// Top-K kernel
// ---------------------------------------------------------------------------
// Shared memory: BATCH staged surfels as 4 x float4 (adjugate rows with the
// local origin and det; opacity and colour) and a per-surfel mask of the
// warps (8 x 4 pixel blocks) that its binning ellipse reaches.  Phase 2
// reuses the area.
//
// The K-set of a pixel lives in registers as an array sorted by decreasing
// weight.  A new weight runs down a compare-exchange chain (strictly
// greater moves ahead, so between equal weights the earlier surfel stays
// in front and the later one is the first to fall off the end).  For K <
// KCAP the first KCAP - K slots hold +inf and never move, so the K-th
// largest weight is always slot KCAP - 1.  With the first-K selection the
// K slots after the padding take the first K contributors in order.
template <int TS, int KCAP, typename FT, bool FRONT, bool AUX, bool LOSS = false, bool SORT = false>
__global__ void __launch_bounds__(TS * TS, KCAP <= 8 ? 1024 / (TS * TS) : (KCAP == 16 && TS <= 16 ? 512 / (TS * TS) : 1)) k_render_topk(const __grid_constant__ Cams cams,
                                                         const __grid_constant__ RParams P, const FwdArgs a,
                                                         const __grid_constant__ AuxOut x) {
    constexpr int NT = TS * TS;
    constexpr int PC = (NT < 65536 / (KCAP * 8 + 4)) ? NT : 65536 / (KCAP * 8 + 4);  // phase-2 pixel chunk
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_r0 = reinterpret_cast<float4*>(smem);
    float4* s_r1 = s_r0 + BATCH;
    float4* s_r2 = s_r1 + BATCH;
    float4* s_oc = s_r2 + BATCH;                                 // (o, r, g, b)
    uint32_t* s_wm = reinterpret_cast<uint32_t*>(s_oc + BATCH);  // warps the footprint reaches
    float4* s_nrm = reinterpret_cast<float4*>(s_wm + BATCH);     // AUX: facing normals
    int32_t* s_id = reinterpret_cast<int32_t*>(smem);            // phase 2: [PC][KCAP] ids
    float* s_w = reinterpret_cast<float*>(s_id + PC * KCAP);     //          [PC][KCAP] weights
    int32_t* s_n = reinterpret_cast<int32_t*>(s_w + PC * KCAP);
    unsigned long long* s_lab =  // AUX: per-pixel argmax keys
        reinterpret_cast<unsigned long long*>(smem + (((size_t)PC * KCAP * 8 + PC * 4 + 7) & ~(size_t)7));
    __shared__ int s_tile;
    __shared__ uint32_t s_bits[NT / 32][BATCH / 32];  // per warp: the staged surfels its block meets
    __shared__ float s_loss[LOSS ? NT / 32 : 1];        // LOSS: per-warp sums of a tile

    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t wbit = 1u << (tid >> 5);
    if (a.st->err) return;
    const int K = P.K;
    const FT* __restrict__ feats = reinterpret_cast<const FT*>(a.feats);
    constexpr int E = FeatVec<FT>::E;
    const int nvec = P.C / E;
    const int ppi = NT / nvec;                         // pixels per phase-2 sweep
    const int q0 = tid / nvec, vv = tid - q0 * nvec;   // this thread's pixel offset and 16-byte chunk
    for (int t = next_tile(cams, a, &s_tile, true); t < cams.total_tiles; t = next_tile(cams, a, &s_tile, false)) {
        if constexpr (SORT) {  // this tile's depth sort first, in the staging area
            __syncthreads();   // (the previous tile's last reads of the area)
            sort_tile(cams, P, a.rec, x.sort.binrec, a.ranges, x.sort.list, x.sort.unb_list, x.sort.scratch,
                      x.sort.masks, a.st, t, reinterpret_cast<uint64_t*>(smem),
                      reinterpret_cast<uint32_t*>(smem + (size_t)SORT_CAP * 8),
                      reinterpret_cast<uint16_t*>(smem + (size_t)SORT_CAP * 12));
            __syncthreads();  // the sorted list and masks (global, written by this CTA) before staging
        }
        const int view = view_of_tile(cams, t);
        const CamDev& cam = cams.c[view];
        const int lt = t - cam.tile_off;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        const int2 lp = pixel_of<TS>(tid);
        const int px = tx * TS + lp.x, py = ty * TS + lp.y;
        const bool inside = px < cam.W && py < cam.H;
        const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
        const int2 rg = checked_range(a.ranges, t, P.pair_cap, a.st);
        const int n = rg.y - rg.x;
        const int64_t vbase = (int64_t)view * P.N;
        const float* __restrict__ rgbv = a.rgb + (P.color_sh ? 3 * vbase : 0);  // SH: item colours
        if (LOSS && inside) {  // the pixel's targets, into L2 while phase 1 runs
            const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
            const char* ft = reinterpret_cast<const char*>(x.loss.Ft) + pix * P.C * (int64_t)sizeof(FT);
            for (int off = 0; off < P.C * (int)sizeof(FT); off += 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(ft + off));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(x.loss.rgbt + 3 * pix));
        }

        float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        bool done = !inside;
        int last = -1;
        float hw[KCAP];
        int hp[KCAP];
#pragma unroll
        for (int k = 0; k < KCAP; ++k) {
            hw[k] = k < KCAP - K ? INFINITY : -INFINITY;
            hp[k] = -1;
        }
        uint32_t n_eval = 0, n_contrib = 0;
        int n_sel = 0;  // FRONT: contributors taken so far
        float zs = 0.0f, zmed = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;  // AUX sums
        bool med = false;

        for (int b0 = 0; b0 < n; b0 += BATCH) {
            if (__syncthreads_and(done)) break;
            const int cnt = min(BATCH, n - b0);
            for (int j = tid; j < cnt; j += NT) {
                const uint32_t item = a.list[rg.x + b0 + j];
                if (!in_bounds(a.st, SITE_ITEM, (int64_t)item - vbase, P.N)) {  // check build: a dead record
                    s_oc[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    s_wm[j] = 0u;
                    continue;
                }
                const float4* r = a.rec + 4 * (size_t)item;
                s_r0[j] = r[0];
                s_r1[j] = r[1];
                s_r2[j] = r[2];
                const int64_t sp = (int64_t)item - vbase;
                s_oc[j] = make_float4(r[3].x, rgbv[3 * sp], rgbv[3 * sp + 1], rgbv[3 * sp + 2]);
                s_wm[j] = a.masks[rg.x + b0 + j];
                if (a.out_feat) {  // the feature row, into L2 while phase 1 runs (phase 2 gathers the selected ones)
                    const char* row = reinterpret_cast<const char*>(feats + (size_t)sp * P.C);
                    for (int off = 0; off < P.C * (int)sizeof(FT); off += 128)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(row + off));
                }
                if (AUX) {  // facing normal, and the centre depth for the low-pass screen term
                    const float4 nf = facing_normal(r[2], r[0].w, r[1].w, cam);
                    s_nrm[j] = make_float4(nf.x, nf.y, nf.z, r[3].y);
                }
            }
            __syncthreads();
            // this warp's staged surfels as bit words (the footprint misses the
            // other ones): the loop below visits set bits only
#pragma unroll
            for (int i = 0; i < BATCH / 32; ++i) {
                const int j = 32 * i + lane;
                const uint32_t word = __ballot_sync(0xffffffffu, j < cnt && (s_wm[j] & wbit));
                if (lane == i) s_bits[tid >> 5][i] = word;
            }
            __syncwarp();
            if (done) continue;
            for (int i = 0; i < (cnt + 31) >> 5 && !done; ++i) {
            for (uint32_t bits = s_bits[tid >> 5][i]; bits != 0u; bits &= bits - 1u) {
                const int j = 32 * i + __ffs(bits) - 1;
                ++n_eval;
                Hit h;
                const float4 oc = s_oc[j];
                if (!eval_splat<AUX>(s_r0[j], s_r1[j], s_r2[j], oc.x, pxf, pyf, P.alpha_min, cam.near_plane, h, P.lowpass))
                    continue;
                const float alpha = fminf(h.alpha_raw, P.alpha_max);
                const float Tn = T * (1.0f - alpha);
                if (Tn < P.T_min) { done = true; break; }
                const float w = alpha * T;
                cr = fmaf(w, oc.y, cr);
                cg = fmaf(w, oc.z, cg);
                cb = fmaf(w, oc.w, cb);
                ++n_contrib;
                if (AUX) {
                    const float4 nv = s_nrm[j];
                    const float zh = h.scr ? nv.w : s_r2[j].w * h.inv;  // hit depth, as in the near-plane test
                    zs = fmaf(w, zh, zs);
                    nx = fmaf(w, nv.x, nx);
                    ny = fmaf(w, nv.y, ny);
                    nz = fmaf(w, nv.z, nz);
                    if (!med && Tn < 0.5f) { zmed = zh; med = true; }
                }
                if (FRONT) {
                    // the first K contributors, in the K slots after the padding
                    if (n_sel < K) {
                        const int slot = KCAP - K + n_sel;
#pragma unroll
                        for (int k = 0; k < KCAP; ++k) {
                            hw[k] = k == slot ? w : hw[k];
                            hp[k] = k == slot ? b0 + j : hp[k];
                        }
                        ++n_sel;
                    }
                } else if (w > hw[KCAP - 1]) {
                    float x = w;
                    int xp = b0 + j;
#pragma unroll
                    for (int k = 0; k < KCAP; ++k) {
                        const bool gt = x > hw[k];
                        const float nw = gt ? x : hw[k];
                        const int np = gt ? xp : hp[k];
                        x = gt ? hw[k] : x;
                        xp = gt ? hp[k] : xp;
                        hw[k] = nw;
                        hp[k] = np;
                    }
                }
                T = Tn;
                last = b0 + j;
                if (P.stop_rule == FSS_STOP_EXACT_TOPK && (FRONT ? n_sel == K : P.alpha_max * T <= hw[KCAP - 1])) {
                    done = true;
                    break;
                }
            }
            }
        }

        // per-pixel outputs; the K-set in front-to-back order
        float lsum = 0.0f;  // LOSS: this thread's weighted loss terms in this tile (nothing live in phase 1)
        float rt[3] = {0.0f, 0.0f, 0.0f};  // LOSS: the colour target, loaded ahead of the ranks
        if (LOSS && inside) {
            const float* r = x.loss.rgbt + 3 * (cam.pix_off + (int64_t)py * cam.W + px);
#pragma unroll
            for (int c = 0; c < 3; ++c) rt[c] = __ldcs(r + c);
        }
        int rank[KCAP], hid[KCAP];
        int hc = 0;
#pragma unroll
        for (int k = 0; k < KCAP; ++k) {
            hc += hp[k] >= 0 ? 1 : 0;
            int r = 0;
#pragma unroll
            for (int j = 0; j < KCAP; ++j) r += (hp[j] >= 0 && hp[j] < hp[k]) ? 1 : 0;
            rank[k] = r;
        }
        const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
        if (inside) {
            if (a.out_rgb) {
                a.out_rgb[3 * pix] = fmaf(T, P.bg[0], cr);
                a.out_rgb[3 * pix + 1] = fmaf(T, P.bg[1], cg);
                a.out_rgb[3 * pix + 2] = fmaf(T, P.bg[2], cb);
                if (LOSS) {  // the colour term: |rgb - rgb_t| and its sign
                    const float c3[3] = {fmaf(T, P.bg[0], cr), fmaf(T, P.bg[1], cg), fmaf(T, P.bg[2], cb)};
                    float s1 = 0.0f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float d = c3[c] - rt[c];
                        s1 += fabsf(d);
                        x.loss.drgb[3 * pix + c] = d > 0.0f ? x.loss.sc : (d < 0.0f ? -x.loss.sc : 0.0f);
                    }
                    lsum = fmaf(x.loss.sc, s1, lsum);
                }
            }
            if (a.out_T) a.out_T[pix] = T;
            if (a.saved_nstop) a.saved_nstop[pix] = last + 1;
            if (AUX) {
                if (x.depth) x.depth[pix] = zs;
                if (x.depth_med) x.depth_med[pix] = zmed;
                if (x.normal) {
                    x.normal[3 * pix] = nx;
                    x.normal[3 * pix + 1] = ny;
                    x.normal[3 * pix + 2] = nz;
                }
            }
#pragma unroll
            for (int k = 0; k < KCAP; ++k) {
                hid[k] = -1;
                if (hp[k] >= 0) {
                    const int64_t o = pix * K + rank[k];
                    hid[k] = (int32_t)((int64_t)a.list[rg.x + hp[k]] - vbase);
                    if (a.out_ids) a.out_ids[o] = hid[k];
                    if (a.saved_pos) a.saved_pos[o] = hp[k];
                    if (a.saved_w) a.saved_w[o] = hw[k];
                }
            }
            for (int k = hc; k < K; ++k) {
                const int64_t o = pix * K + k;
                if (a.out_ids) a.out_ids[o] = -1;
                if (a.saved_pos) a.saved_pos[o] = -1;
                if (a.saved_w) a.saved_w[o] = 0.0f;
            }
        }
        warp_count(&a.st->counters[0], n_eval);
        warp_count(&a.st->counters[1], n_contrib);

        // phase 2: gather-accumulate the selected feature rows (AUX: and their argmax)
        if (a.out_feat || (AUX && x.label)) {
            for (int p0 = 0; p0 < NT; p0 += PC) {
                __syncthreads();
                if (tid >= p0 && tid < p0 + PC) {
                    const int q = tid - p0;
                    s_n[q] = inside ? hc : 0;
                    if (AUX) s_lab[q] = 0ull;
                    float wsc = 1.0f;  // renormalised variant: 1 / (sum of the selected weights)
                    if (P.renorm) {
                        float ws = 0.0f;
#pragma unroll
                        for (int k = 0; k < KCAP; ++k) ws += hp[k] >= 0 ? hw[k] : 0.0f;
                        wsc = ws > 0.0f ? __frcp_rn(ws) : 0.0f;
                    }
#pragma unroll
                    for (int k = 0; k < KCAP; ++k) {
                        if (hp[k] >= 0) {
                            s_id[q * KCAP + rank[k]] = hid[k];
                            s_w[q * KCAP + rank[k]] = hw[k] * wsc;
                        }
                    }
                }
                __syncthreads();
                const int npx = min(PC, NT - p0);
                for (int q = q0; q0 < ppi && q < npx; q += ppi) {
                    const int p = p0 + q;
                    const int2 lq = pixel_of<TS>(p);  // pixel of the thread that selected row q
                    const int qx = tx * TS + lq.x, qy = ty * TS + lq.y;
                    if (qx >= cam.W || qy >= cam.H) continue;
                    typename FeatVec<FT>::Raw ft{};  // LOSS: the target chunk, loaded during the gathers
                    if (LOSS)
                        ft = FeatVec<FT>::raw_cs(reinterpret_cast<const FT*>(x.loss.Ft) +
                                                 (cam.pix_off + (int64_t)qy * cam.W + qx) * P.C + vv * E);
                    // the selected rows' chunks, weighted with packed FP32 pairs (lane for
                    // lane fmaf) in the selection's front-to-back order
                    float2 acc2[E / 2];
#pragma unroll
                    for (int e = 0; e < E / 2; ++e) acc2[e] = make_float2(0.0f, 0.0f);
                    const int c = s_n[q];
                    for (int k = 0; k < c; ++k) {
                        const int id = s_id[q * KCAP + k];
                        const float w = s_w[q * KCAP + k];
                        if (!in_bounds(a.st, SITE_FEAT_ROW, id, P.N)) continue;
                        float2 f2[E / 2];
                        FeatVec<FT>::unpack2(FeatVec<FT>::raw(feats + (size_t)id * P.C + vv * E), f2);
                        const float2 w2 = make_float2(w, w);
#pragma unroll
                        for (int e = 0; e < E / 2; ++e) acc2[e] = __ffma2_rn(w2, f2[e], acc2[e]);
                    }
                    const int64_t qpix = cam.pix_off + (int64_t)qy * cam.W + qx;
                    if constexpr (LOSS) {
                        // F as stored (output type = feature type), then the feature term:
                        // d = F - F_t (an FMA with -1: one rounding, as the subtraction),
                        // sum d^2, dL/dF = sf d rounded once to the output type
                        // (F with an evict-first store: the step does not read it again)
                        using Raw = typename FeatVec<FT>::Raw;
                        const Raw fr = FeatVec<FT>::pack(acc2);
                        __stcs(reinterpret_cast<Raw*>(reinterpret_cast<FT*>(a.out_feat) + qpix * P.C + vv * E), fr);
                        float2 f2[E / 2], t2[E / 2], g2[E / 2];
                        FeatVec<FT>::unpack2(fr, f2);
                        FeatVec<FT>::unpack2(ft, t2);
                        const float2 m1 = make_float2(-1.0f, -1.0f), sf2 = make_float2(x.loss.sf, x.loss.sf);
                        float2 q2 = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int e = 0; e < E / 2; ++e) {
                            const float2 d2 = __ffma2_rn(t2[e], m1, f2[e]);
                            q2 = __ffma2_rn(d2, d2, q2);
                            g2[e] = __fmul2_rn(sf2, d2);
                        }
                        FeatVec<FT>::st(reinterpret_cast<FT*>(x.loss.dF) + qpix * P.C + vv * E, FeatVec<FT>::pack(g2));
                        lsum = fmaf(x.loss.lf, q2.x + q2.y, lsum);
                    } else {
                        float acc[E];
#pragma unroll
                        for (int e = 0; e < E / 2; ++e) {
                            acc[2 * e] = acc2[e].x;
                            acc[2 * e + 1] = acc2[e].y;
                        }
                        if (a.out_feat) store_vec<E>(a.out_feat, qpix * P.C + vv * E, acc, P.out_dtype);
                        if (AUX && x.label) {
                            int eb = 0;
                            float bv = acc[0];
#pragma unroll
                            for (int e = 1; e < E; ++e) {
                                eb = acc[e] > bv ? e : eb;
                                bv = acc[e] > bv ? acc[e] : bv;
                            }
                            atomicMax(&s_lab[q], argmax_key(bv, vv * E + eb));
                        }
                    }
                }
                if (AUX && x.label) {
                    __syncthreads();
                    if (tid < npx) {
                        const int2 lq = pixel_of<TS>(p0 + tid);
                        const int qx = tx * TS + lq.x, qy = ty * TS + lq.y;
                        if (qx < cam.W && qy < cam.H)
                            x.label[cam.pix_off + (int64_t)qy * cam.W + qx] =
                                s_n[tid] > 0 ? argmax_channel(s_lab[tid]) : -1;
                    }
                }
            }
        }
        if constexpr (LOSS) {  // the tile's share of the loss, one double atomic per tile
            float v = lsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s_loss[tid >> 5] = v;
            __syncthreads();  // (the next tile's writes come after its own barriers)
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < NT / 32; ++w) t += s_loss[w];
                atomicAdd(x.loss.loss, t);
            }
        }
    }
}

template <int TS, typename FT>
cudaError_t launch_topk(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                        cudaStream_t s) {
    constexpr int NT = TS * TS;
    const bool aux = x.any() || P.lowpass;  // the variant instances also carry the low-pass filter
    auto smem = [aux](int kcap) {
        const size_t p1 = (size_t)BATCH * (4 * 16 + 4) + (aux ? (size_t)BATCH * 16 : 0);  // staging (+ normals)
        const int pc = (NT < 65536 / (kcap * 8 + 4)) ? NT : 65536 / (kcap * 8 + 4);
        return std::max(p1, (size_t)pc * (kcap * 8 + 4) + (aux ? (size_t)pc * 8 + 8 : 0));  // (+ argmax keys)
    };
    // the fused loss (and sort): the plain selection with K <= 8, no sensor outputs (checked by the caller)
    if (x.loss.loss && x.sort.list)
        return launch_tiles(k_render_topk<TS, 8, FT, false, false, true, true>, NT,
                            std::max(smem(8), SORT_SMEM_BYTES), cams, P, a, x, num_sms, s);
    if (x.loss.loss)
        return launch_tiles(k_render_topk<TS, 8, FT, false, false, true>, NT, smem(8), cams, P, a, x, num_sms, s);
    // variants (first-K selection, sensor outputs) need unsorted or few slots: two capacities
    if (P.select == FSS_SELECT_FRONT) {
        if (aux) {
            if (P.K <= 8) return launch_tiles(k_render_topk<TS, 8, FT, true, true>, NT, smem(8), cams, P, a, x, num_sms, s);
            return launch_tiles(k_render_topk<TS, 32, FT, true, true>, NT, smem(32), cams, P, a, x, num_sms, s);
        }
        if (P.K <= 8) return launch_tiles(k_render_topk<TS, 8, FT, true, false>, NT, smem(8), cams, P, a, x, num_sms, s);
        return launch_tiles(k_render_topk<TS, 32, FT, true, false>, NT, smem(32), cams, P, a, x, num_sms, s);
    }
    if (aux) {
        if (P.K <= 8) return launch_tiles(k_render_topk<TS, 8, FT, false, true>, NT, smem(8), cams, P, a, x, num_sms, s);
        return launch_tiles(k_render_topk<TS, 32, FT, false, true>, NT, smem(32), cams, P, a, x, num_sms, s);
    }
    if (P.K <= 4) return launch_tiles(k_render_topk<TS, 4, FT, false, false>, NT, smem(4), cams, P, a, x, num_sms, s);
    if (P.K <= 8) return launch_tiles(k_render_topk<TS, 8, FT, false, false>, NT, smem(8), cams, P, a, x, num_sms, s);
    if (P.K <= 16) return launch_tiles(k_render_topk<TS, 16, FT, false, false>, NT, smem(16), cams, P, a, x, num_sms, s);
    return launch_tiles(k_render_topk<TS, 32, FT, false, false>, NT, smem(32), cams, P, a, x, num_sms, s);
}

template <typename FT>
cudaError_t launch_topk_dtype(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                              cudaStream_t s) {
    if (P.ts == 8) return launch_topk<8, FT>(cams, P, a, x, num_sms, s);
    if (P.ts == 16) return launch_topk<16, FT>(cams, P, a, x, num_sms, s);
    return launch_topk<32, FT>(cams, P, a, x, num_sms, s);
}

}  // namespace fss
