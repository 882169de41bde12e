// Full-accumulation forward render (K = 0, the plain path of Eq. 2): the
// same traversal as the Top-K kernel, but every batch stages the feature rows
// of its surfels in shared memory and each contributor adds w c_i over all C
// channels in registers.
#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"

#include <algorithm>
#include <climits>

namespace fss {

namespace {

__device__ __forceinline__ int next_tile(const Cams& cams, const FwdArgs& a, int* s_tile, bool first) {
    return next_tile_q(a.persistent, &a.st->work, s_tile, first, cams);
}

}  // namespace

// ---------------------------------------------------------------------------
// full-accumulation kernel (K = 0): all contributors, all channels
// ---------------------------------------------------------------------------
template <int TS, int CMAX, typename FT, bool AUX>
__global__ void __launch_bounds__(TS * TS) k_render_full(const __grid_constant__ Cams cams,
                                                         const __grid_constant__ RParams P, const FwdArgs a,
                                                         const __grid_constant__ AuxOut x) {
    constexpr int NT = TS * TS;
    constexpr int E = FeatVec<FT>::E;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_r0 = reinterpret_cast<float4*>(smem);
    float4* s_r1 = s_r0 + FBATCH;
    float4* s_r2 = s_r1 + FBATCH;
    float4* s_oc = s_r2 + FBATCH;                                   // (o, r, g, b)
    uint32_t* s_wm = reinterpret_cast<uint32_t*>(s_oc + FBATCH);    // warps the footprint reaches
    float* s_f = reinterpret_cast<float*>(s_wm + 2 * FBATCH);       // [FBATCH][C] f32 (16-byte aligned)
    float4* s_nrm = reinterpret_cast<float4*>(s_f + (size_t)FBATCH * P.C);  // AUX: facing normals
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    if (a.st->err) return;
    const int C = P.C;
    const FT* __restrict__ feats = reinterpret_cast<const FT*>(a.feats);
    const uint32_t wbit = 1u << (tid >> 5);
    const int nv = C / E;
    const int rpi = NT / nv;                         // staged rows per sweep
    const int r0 = tid / nv, vv0 = tid - r0 * nv;    // this thread's row offset and 16-byte chunk
    for (int t = next_tile(cams, a, &s_tile, true); t < cams.total_tiles; t = next_tile(cams, a, &s_tile, false)) {
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

        float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        float acc[CMAX];
#pragma unroll
        for (int c = 0; c < CMAX; ++c) acc[c] = 0.0f;
        bool done = !inside;
        int last = -1;
        uint32_t n_eval = 0, n_contrib = 0;
        float zs = 0.0f, zmed = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;  // AUX sums
        bool med = false;

        for (int b0 = 0; b0 < n; b0 += FBATCH) {
            if (__syncthreads_and(done)) break;
            const int cnt = min(FBATCH, n - b0);
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
                if (AUX) {  // facing normal, and the centre depth for the low-pass screen term
                    const float4 nf = facing_normal(r[2], r[0].w, r[1].w, cam);
                    s_nrm[j] = make_float4(nf.x, nf.y, nf.z, r[3].y);
                }
            }
            if (r0 < rpi) {
                for (int j = r0; j < cnt; j += rpi) {
                    const int64_t sp = (int64_t)a.list[rg.x + b0 + j] - vbase;
                    if (!FSS_CHECKED(sp >= 0 && sp < P.N)) continue;  // recorded by the staging loop
                    float f[E];
                    FeatVec<FT>::load(feats + (size_t)sp * C + vv0 * E, f);
#pragma unroll
                    for (int e = 0; e < E; ++e) s_f[j * C + vv0 * E + e] = f[e];
                }
            }
            __syncthreads();
            if (done) continue;
            for (int j = 0; j < cnt; ++j) {
                if (!(s_wm[j] & wbit)) continue;  // warp-uniform
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
                const float4* fr = reinterpret_cast<const float4*>(s_f + j * C);
#pragma unroll
                for (int c4 = 0; c4 < CMAX / 4; ++c4) {
                    if (4 * c4 < C) {
                        const float4 f = fr[c4];
                        acc[4 * c4] = fmaf(w, f.x, acc[4 * c4]);
                        acc[4 * c4 + 1] = fmaf(w, f.y, acc[4 * c4 + 1]);
                        acc[4 * c4 + 2] = fmaf(w, f.z, acc[4 * c4 + 2]);
                        acc[4 * c4 + 3] = fmaf(w, f.w, acc[4 * c4 + 3]);
                    }
                }
                T = Tn;
                last = b0 + j;
            }
        }
        if (inside) {
            const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
            if (a.out_rgb) {
                a.out_rgb[3 * pix] = fmaf(T, P.bg[0], cr);
                a.out_rgb[3 * pix + 1] = fmaf(T, P.bg[1], cg);
                a.out_rgb[3 * pix + 2] = fmaf(T, P.bg[2], cb);
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
                if (x.label) {  // argmax over the channels, lowest index on ties
                    int cb = 0;
                    float bv = acc[0];
#pragma unroll
                    for (int c = 1; c < CMAX; ++c) {
                        const bool gt = c < C && acc[c] > bv;
                        cb = gt ? c : cb;
                        bv = gt ? acc[c] : bv;
                    }
                    x.label[pix] = n_contrib > 0 ? cb : -1;
                }
            }
            if (a.out_feat) {
#pragma unroll
                for (int c4 = 0; c4 < CMAX / 4; ++c4)
                    if (4 * c4 < C) store_vec<4>(a.out_feat, pix * C + 4 * c4, &acc[4 * c4], P.out_dtype);
            }
        }
        warp_count(&a.st->counters[0], n_eval);
        warp_count(&a.st->counters[1], n_contrib);
    }
}

namespace {

template <int TS, typename FT>
cudaError_t launch_full(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms, cudaStream_t s) {
    constexpr int NT = TS * TS;
    const bool aux = x.any() || P.lowpass;  // the variant instances also carry the low-pass filter
    const size_t smem = (size_t)FBATCH * (4 * 16 + 8) + (size_t)FBATCH * P.C * 4 +
                        (aux ? (size_t)FBATCH * 16 : 0);  // staging, masks, rows (+ normals)
#define FSS_FULL(CM)                                                                                         \
    return aux ? launch_tiles(k_render_full<TS, CM, FT, true>, NT, smem, cams, P, a, x, num_sms, s)           \
               : launch_tiles(k_render_full<TS, CM, FT, false>, NT, smem, cams, P, a, x, num_sms, s)
    if (P.C <= 16) FSS_FULL(16);
    if (P.C <= 32) FSS_FULL(32);
    if (P.C <= 64) FSS_FULL(64);
    FSS_FULL(128);
#undef FSS_FULL
}

template <typename FT>
cudaError_t launch_full_dtype(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                              cudaStream_t s) {
    if (P.ts == 8) return launch_full<8, FT>(cams, P, a, x, num_sms, s);
    if (P.ts == 16) return launch_full<16, FT>(cams, P, a, x, num_sms, s);
    return launch_full<32, FT>(cams, P, a, x, num_sms, s);
}

}  // namespace

cudaError_t launch_render_full(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                               cudaStream_t s) {
    if (P.feat_dtype == FSS_BF16) return launch_full_dtype<__nv_bfloat16>(cams, P, a, x, num_sms, s);
    return launch_full_dtype<float>(cams, P, a, x, num_sms, s);
}

}  // namespace fss
