// Backward render for sm_103a: vector-Jacobian product of the forward
// render (Eq. 2, Eq. 7) with the Top-K set, skips, stops and clamps held
// fixed.  The paper trains through the renderer end to end (Sec. 3.1
// "differentiable", Sec. 3.5) but prints no gradients; these are the chain
// rule of the forward:
//   s_j    = rgb_j . dL/dRGB + [j in K-set] c_j . dL/dF
//   dL/da_j = T_j (s_j - S_j),  S_j = sum_{i>j} w_i s_i / T_{j+1} + bg.dL/dRGB + dL/dT
//   S_{j-1} = a_j s_j + (1 - a_j) S_j,  T_j = T_{j+1} / (1 - a_j)
// replayed back to front from the saved traversal length and final T.
//
// k_bwd_feat  (Top-K) one CTA per tile: for every selected (pixel, k) the
//             dot c_i . dL/dF(x) and the feature gradient sum w_i dL/dF(x),
//             grouped by surfel in shared memory first, so each surfel costs
//             one row of 16-byte vector reductions per tile.
// k_bwd_geo   one CTA per tile, one thread per pixel: back-to-front replay;
//             per staged surfel the warp reduce-scatters its 13 partial
//             derivatives (adjugate rows 9, opacity 1, colour 3) and the
//             CTA flushes one row of vector reductions per surfel and tile.
//             The full-accumulation variant also forms c_j . dL/dF inline
//             and reduce-scatters the feature gradient.
// k_bwd_project one thread per surfel: adjugate-row gradients -> homography
//             columns -> means, scales, quaternions; sums the views.
// k_feat_out  writes every row of the feature gradient (zeros for surfels
//             culled in every view).
#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"

#include <algorithm>
#include <climits>

namespace fss {

namespace {

constexpr int BB = 128;      // staged surfels per backward batch
constexpr int PCAP = 2048;   // list positions per k_bwd_feat pass
constexpr int BWD_FEAT_THREADS = 256;

// reduce-scatter of V values (power of two, 2..32 per lane...) across a warp:
// afterwards lane l holds the warp sum of values (V/32)*l + i for V >= 32, or
// of value l >> (5 - log2 V) for V < 32 (lanes sharing it hold equal sums).
template <int V>
__device__ __forceinline__ void reduce_scatter(float* v) {
    const int lane = threadIdx.x & 31;
    int n = V;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (n > 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < V / 2; ++i) {
                if (i < n / 2) {
                    const float send = up ? v[i] : v[i + n / 2];
                    const float keep = up ? v[i + n / 2] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            n >>= 1;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// ---------------------------------------------------------------------------
// k_bwd_feat (Top-K): dots and feature gradients, grouped per tile
// ---------------------------------------------------------------------------
template <int CPL, typename FT>
__global__ void __launch_bounds__(BWD_FEAT_THREADS) k_bwd_feat(const __grid_constant__ Cams cams,
                                                              const __grid_constant__ RParams P, const BwdArgs a,
                                                              int ucap) {
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t* s_slot = reinterpret_cast<int32_t*>(smem);  // [PCAP] flag -> slot
    int32_t* s_inv = s_slot + PCAP;                      // [PCAP] slot -> position
    float* s_feat = reinterpret_cast<float*>(s_inv + PCAP);  // [ucap][C]
    float* s_acc = s_feat + (size_t)ucap * P.C;              // [ucap][C]
    __shared__ int s_red[32];
    __shared__ int s_max;

    if (a.st->err) return;
    const int t = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int K = P.K, C = P.C, ts = P.ts, npx = ts * ts;
    const int view = view_of_tile(cams, t);
    const CamDev& cam = cams.c[view];
    const int lt = t - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int2 rg = a.ranges[t];
    const int64_t vbase = (int64_t)view * P.N;
    const FT* __restrict__ feats = reinterpret_cast<const FT*>(a.feats);
    const FT* __restrict__ dF = reinterpret_cast<const FT*>(a.d_feat);

    // longest selected position + 1 over the tile's pixels
    if (tid == 0) s_max = 0;
    __syncthreads();
    int lmax = 0;
    for (int p = tid; p < npx; p += BWD_FEAT_THREADS) {
        const int px = tx * ts + p % ts, py = ty * ts + p / ts;
        if (px >= cam.W || py >= cam.H) continue;
        const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
        for (int k = K - 1; k >= 0; --k) {
            const int pos = a.saved_pos[pix * K + k];
            if (pos >= 0) { lmax = max(lmax, pos + 1); break; }
        }
    }
    atomicMax(&s_max, lmax);
    __syncthreads();
    const int L = s_max;

    for (int p0 = 0; p0 < L; p0 += PCAP) {
        for (int i = tid; i < PCAP; i += BWD_FEAT_THREADS) s_slot[i] = 0;
        __syncthreads();
        for (int p = tid; p < npx; p += BWD_FEAT_THREADS) {
            const int px = tx * ts + p % ts, py = ty * ts + p / ts;
            if (px >= cam.W || py >= cam.H) continue;
            const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
            for (int k = 0; k < K; ++k) {
                const int pos = a.saved_pos[pix * K + k];
                if (pos >= p0 && pos < p0 + PCAP) s_slot[pos - p0] = 1;
            }
        }
        __syncthreads();
        // exclusive scan of the flags (PCAP / 256 = 8 per thread)
        constexpr int PER = PCAP / BWD_FEAT_THREADS;
        int f[PER], sum = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) { f[k] = s_slot[tid * PER + k]; sum += f[k]; }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_red[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int w = lane < BWD_FEAT_THREADS / 32 ? s_red[lane] : 0;
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < BWD_FEAT_THREADS / 32) s_red[lane] = wi - w;
            if (lane == BWD_FEAT_THREADS / 32 - 1) s_red[31] = wi;  // total
        }
        __syncthreads();
        int run = s_red[wid] + incl - sum;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int pos = tid * PER + k;
            if (f[k]) { s_slot[pos] = run; s_inv[run] = pos; ++run; }
            else s_slot[pos] = -1;
        }
        __syncthreads();
        const int U = s_red[31];

        for (int u0 = 0; u0 < U; u0 += ucap) {
            const int u1 = min(U, u0 + ucap);
            // stage the feature rows of slots [u0, u1) and clear their accumulators
            for (int idx = tid; idx < (u1 - u0) * C; idx += BWD_FEAT_THREADS) {
                const int sl = idx / C, ch = idx - sl * C;
                const int64_t sp = (int64_t)a.list[rg.x + p0 + s_inv[u0 + sl]] - vbase;
                s_feat[idx] = FeatVec<FT>::one(feats + sp * C + ch);
                s_acc[idx] = 0.0f;
            }
            __syncthreads();
            // one warp per pixel: dL/dF row in registers, then its entries
            for (int p = wid; p < npx; p += BWD_FEAT_THREADS / 32) {
                const int px = tx * ts + p % ts, py = ty * ts + p / ts;
                if (px >= cam.W || py >= cam.H) continue;
                const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
                int pos = -1;
                float w = 0.0f;
                int sl = -1;
                if (lane < K) {
                    pos = a.saved_pos[pix * K + lane];
                    w = a.saved_w[pix * K + lane];
                    if (pos >= p0 && pos < p0 + PCAP) {
                        const int s2 = s_slot[pos - p0];
                        if (s2 >= u0 && s2 < u1) sl = s2 - u0;
                    }
                }
                unsigned rel = __ballot_sync(0xffffffffu, sl >= 0);
                if (!rel) continue;
                float df[CPL];
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int ch = lane + 32 * i;
                    df[i] = ch < C ? FeatVec<FT>::one(dF + pix * C + ch) : 0.0f;
                }
                while (rel) {
                    const int k = __ffs(rel) - 1;
                    rel &= rel - 1;
                    const int slk = __shfl_sync(0xffffffffu, sl, k);
                    const float wk = __shfl_sync(0xffffffffu, w, k);
                    float dot = 0.0f;
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const int ch = lane + 32 * i;
                        if (ch < C) {
                            dot = fmaf(s_feat[slk * C + ch], df[i], dot);
                            atomicAdd(&s_acc[slk * C + ch], wk * df[i]);
                        }
                    }
                    dot = warp_sum(dot);
                    if (lane == 0) a.dots[pix * K + k] = dot;
                }
            }
            __syncthreads();
            // flush: one row of 16-byte reductions per surfel
            const int c4 = C / 4;
            for (int idx = tid; idx < (u1 - u0) * c4; idx += BWD_FEAT_THREADS) {
                const int sl = idx / c4, q = idx - sl * c4;
                const int64_t sp = (int64_t)a.list[rg.x + p0 + s_inv[u0 + sl]] - vbase;
                const int slot = a.splat_slot[sp];
                const float* v = s_acc + sl * C + 4 * q;
                red_add_v4(a.feat_acc + (int64_t)slot * C + 4 * q, v[0], v[1], v[2], v[3]);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// k_bwd_geo: back-to-front replay (Top-K and full accumulation)
// ---------------------------------------------------------------------------
template <int TS, bool FULL, int CMAX, typename FT>
__global__ void __launch_bounds__(TS * TS) k_bwd_geo(const __grid_constant__ Cams cams,
                                                     const __grid_constant__ RParams P, const BwdArgs a) {
    constexpr int NT = TS * TS;
    constexpr int NB = FULL ? FBATCH : BB;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_r0 = reinterpret_cast<float4*>(smem);
    float4* s_r1 = s_r0 + NB;
    float4* s_r2 = s_r1 + NB;
    float* s_o = reinterpret_cast<float*>(s_r2 + NB);
    float* s_c0 = s_o + NB;
    float* s_c1 = s_c0 + NB;
    float* s_c2 = s_c1 + NB;
    float* s_g = s_c2 + NB;        // [NB][16] partial derivatives
    float* s_f = s_g + NB * 16;    // FULL: [NB][C] features
    float* s_gf = s_f + (FULL ? NB * P.C : 0);  // FULL: [NB][C] feature gradients
    __shared__ int s_max;

    if (a.st->err) return;
    const int t = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int C = P.C, K = P.K;
    const int view = view_of_tile(cams, t);
    const CamDev& cam = cams.c[view];
    const int lt = t - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * TS + (tid % TS), py = ty * TS + (tid / TS);
    const bool inside = px < cam.W && py < cam.H;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const int2 rg = a.ranges[t];
    const int64_t vbase = (int64_t)view * P.N;
    const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
    const FT* __restrict__ feats = reinterpret_cast<const FT*>(a.feats);

    int nstop = 0;
    float T = 1.0f, gr = 0.0f, gg = 0.0f, gb = 0.0f, Sh = 0.0f;
    int kk = -1, next_pos = -1;
    float next_dot = 0.0f;
    float dfr[FULL ? CMAX : 1];
#pragma unroll
    for (int c = 0; c < (FULL ? CMAX : 1); ++c) dfr[c] = 0.0f;
    if (inside) {
        nstop = a.saved_nstop[pix];
        T = a.out_T[pix];
        gr = a.d_rgb[3 * pix];
        gg = a.d_rgb[3 * pix + 1];
        gb = a.d_rgb[3 * pix + 2];
        Sh = P.bg[0] * gr + P.bg[1] * gg + P.bg[2] * gb + (a.d_T ? a.d_T[pix] : 0.0f);
        if (!FULL) {
            for (kk = K - 1; kk >= 0; --kk)
                if (a.saved_pos[pix * K + kk] >= 0) break;
            if (kk >= 0) {
                next_pos = a.saved_pos[pix * K + kk];
                next_dot = a.dots[pix * K + kk];
            }
        } else {
            const FT* dF = reinterpret_cast<const FT*>(a.d_feat) + pix * C;
#pragma unroll
            for (int c = 0; c < (FULL ? CMAX : 1); ++c) dfr[c] = c < C ? FeatVec<FT>::one(dF + c) : 0.0f;
        }
    }
    if (tid == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, nstop);
    __syncthreads();
    const int L = s_max;

    for (int b_end = L; b_end > 0; b_end -= NB) {
        const int b_start = max(0, b_end - NB);
        const int cnt = b_end - b_start;
        __syncthreads();
        for (int j = tid; j < cnt; j += NT) {
            const uint32_t item = a.list[rg.x + b_start + j];
            const float4* r = a.rec + 4 * (size_t)item;
            s_r0[j] = r[0];
            s_r1[j] = r[1];
            s_r2[j] = r[2];
            s_o[j] = r[3].x;
            const int64_t sp = (int64_t)item - vbase;
            s_c0[j] = a.rgb[3 * sp];
            s_c1[j] = a.rgb[3 * sp + 1];
            s_c2[j] = a.rgb[3 * sp + 2];
        }
        for (int i = tid; i < cnt * 16; i += NT) s_g[i] = 0.0f;
        if (FULL) {
            const int nvec = C / FeatVec<FT>::E;
            for (int it = tid; it < cnt * nvec; it += NT) {
                const int j = it / nvec, vv = it - j * nvec;
                const int64_t sp = (int64_t)a.list[rg.x + b_start + j] - vbase;
                float f[FeatVec<FT>::E];
                FeatVec<FT>::load(feats + sp * C + vv * FeatVec<FT>::E, f);
#pragma unroll
                for (int e = 0; e < FeatVec<FT>::E; ++e) {
                    s_f[j * C + vv * FeatVec<FT>::E + e] = f[e];
                    s_gf[j * C + vv * FeatVec<FT>::E + e] = 0.0f;
                }
            }
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = b_start + j;
            float g[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) g[k] = 0.0f;
            float w = 0.0f;
            bool contrib = false;
            Hit h;
            if (pos < nstop &&
                eval_splat(s_r0[j], s_r1[j], s_r2[j], s_o[j], pxf, pyf, P.alpha_min, cam.near_plane, h)) {
                contrib = true;
                const float alpha = fminf(h.alpha_raw, P.alpha_max);
                const float Tj = T / (1.0f - alpha);
                w = alpha * Tj;
                float s = s_c0[j] * gr + s_c1[j] * gg + s_c2[j] * gb;
                if (!FULL) {
                    if (pos == next_pos) {
                        s += next_dot;
                        --kk;
                        next_pos = kk >= 0 ? a.saved_pos[pix * K + kk] : -1;
                        next_dot = kk >= 0 ? a.dots[pix * K + kk] : 0.0f;
                    }
                } else {
                    const float4* fr = reinterpret_cast<const float4*>(s_f + j * C);
                    float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
                    for (int c4 = 0; c4 < CMAX / 4; ++c4) {
                        if (4 * c4 < C) {
                            const float4 fv = fr[c4];
                            d0 = fmaf(fv.x, dfr[4 * c4], d0);
                            d1 = fmaf(fv.y, dfr[4 * c4 + 1], d1);
                            d0 = fmaf(fv.z, dfr[4 * c4 + 2], d0);
                            d1 = fmaf(fv.w, dfr[4 * c4 + 3], d1);
                        }
                    }
                    s += d0 + d1;
                }
                const float dal = Tj * (s - Sh);
                Sh = fmaf(alpha, s - Sh, Sh);  // a s + (1 - a) S
                g[10] = w * gr;
                g[11] = w * gg;
                g[12] = w * gb;
                if (h.alpha_raw < P.alpha_max) {
                    const float G = h.alpha_raw / s_o[j];
                    g[9] = dal * G;
                    const float drho = -0.5f * alpha * dal;
                    const float du = 2.0f * h.u * drho, dv = 2.0f * h.v * drho;
                    const float gc0 = du * h.inv, gc1 = dv * h.inv, gc2 = -(du * h.u + dv * h.v) * h.inv;
                    g[0] = gc0 * h.X; g[1] = gc0 * h.Y; g[2] = gc0;
                    g[3] = gc1 * h.X; g[4] = gc1 * h.Y; g[5] = gc1;
                    g[6] = gc2 * h.X; g[7] = gc2 * h.Y; g[8] = gc2;
                }
                T = Tj;
            }
            if (__any_sync(0xffffffffu, contrib)) {
                reduce_scatter<16>(g);  // lane l holds value l >> 1
                if ((lane & 1) == 0 && (lane >> 1) < 13) atomicAdd(&s_g[j * 16 + (lane >> 1)], g[0]);
                if (FULL) {
#pragma unroll
                    for (int c0 = 0; c0 < CMAX; c0 += 32) {
                        if (c0 < C) {
                            float gf[32];
#pragma unroll
                            for (int c = 0; c < 32; ++c) gf[c] = w * dfr[c0 + c];
                            reduce_scatter<32>(gf);  // lane l holds channel c0 + l
                            if (c0 + lane < C) atomicAdd(&s_gf[j * C + c0 + lane], gf[0]);
                        }
                    }
                }
            }
        }
        __syncthreads();
        // flush one gradient row per staged surfel
        for (int j = tid; j < cnt; j += NT) {
            const float* v = s_g + 16 * j;
            bool nz = false;
#pragma unroll
            for (int k = 0; k < 13; ++k) nz |= v[k] != 0.0f;
            if (!nz) continue;
            const int64_t sp = (int64_t)a.list[rg.x + b_start + j] - vbase;
            const int slot = a.splat_slot[sp];
            float* dst = a.grad_item + ((int64_t)view * P.N + slot) * GRAD_STRIDE;
            red_add_v4(dst, v[0], v[1], v[2], v[3]);
            red_add_v4(dst + 4, v[4], v[5], v[6], v[7]);
            red_add_v4(dst + 8, v[8], v[9], v[10], v[11]);
            atomicAdd(dst + 12, v[12]);
        }
        if (FULL) {
            const int c4 = C / 4;
            for (int idx = tid; idx < cnt * c4; idx += NT) {
                const int j = idx / c4, q = idx - j * c4;
                const float* v = s_gf + j * C + 4 * q;
                if (v[0] == 0.0f && v[1] == 0.0f && v[2] == 0.0f && v[3] == 0.0f) continue;
                const int64_t sp = (int64_t)a.list[rg.x + b_start + j] - vbase;
                const int slot = a.splat_slot[sp];
                red_add_v4(a.feat_acc + (int64_t)slot * C + 4 * q, v[0], v[1], v[2], v[3]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_bwd_project: per surfel, d(adjugate rows) -> d(means, scales, quats)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bwd_project(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                     const BwdArgs a) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.N) return;
    float gm[3] = {0, 0, 0}, gs[2] = {0, 0}, gq[4] = {0, 0, 0, 0}, go = 0.0f, gc[3] = {0, 0, 0};
    const int slot = a.st->err ? -1 : a.splat_slot[s];
    if (slot >= 0) {
        const float q0 = a.quats[4 * s], q1 = a.quats[4 * s + 1], q2 = a.quats[4 * s + 2], q3 = a.quats[4 * s + 3];
        const float qn = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
        const float w = q0 / qn, x = q1 / qn, y = q2 / qn, z = q3 / qn;
        const float tu[3] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y)};
        const float tv[3] = {2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x)};
        const float su = a.scales[2 * s], sv = a.scales[2 * s + 1];
        const float pm[3] = {a.means[3 * s], a.means[3 * s + 1], a.means[3 * s + 2]};
        float dtu[3] = {0, 0, 0}, dtv[3] = {0, 0, 0};
        for (int v = 0; v < cams.n; ++v) {
            const float* gv = a.grad_item + ((int64_t)v * P.N + slot) * GRAD_STRIDE;
            const float4 g0 = *reinterpret_cast<const float4*>(gv);
            const float4 g1 = *reinterpret_cast<const float4*>(gv + 4);
            const float4 g2 = *reinterpret_cast<const float4*>(gv + 8);
            const float g12 = gv[12];
            go += g2.y;
            gc[0] += g2.z; gc[1] += g2.w; gc[2] += g12;
            if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
                g1.z == 0.f && g1.w == 0.f && g2.x == 0.f)
                continue;
            const CamDev& cam = cams.c[v];
            const float4 r0 = a.rec[4 * ((int64_t)v * P.N + s)], r1 = a.rec[4 * ((int64_t)v * P.N + s) + 1];
            const float4 r3 = a.rec[4 * ((int64_t)v * P.N + s) + 3];
            const float xc = r0.w, yc = r1.w, sc = r3.w;
            // gradient of the unshifted adjugate: sc * G S^T
            const float G[3][3] = {{g0.x, g0.y, g0.z}, {g0.w, g1.x, g1.y}, {g1.z, g1.w, g2.x}};
            float gA[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                gA[r][0] = sc * (G[r][0] + xc * G[r][2]);
                gA[r][1] = sc * (G[r][1] + yc * G[r][2]);
                gA[r][2] = sc * G[r][2];
            }
            // homography columns c0 = K Rv r_u t_u, c1 = K Rv r_v t_v, c2 = K (Rv p + t)
            float eu[3], ev[3], pc[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                eu[r] = cam.R[3 * r] * tu[0] + cam.R[3 * r + 1] * tu[1] + cam.R[3 * r + 2] * tu[2];
                ev[r] = cam.R[3 * r] * tv[0] + cam.R[3 * r + 1] * tv[1] + cam.R[3 * r + 2] * tv[2];
                pc[r] = cam.R[3 * r] * pm[0] + cam.R[3 * r + 1] * pm[1] + cam.R[3 * r + 2] * pm[2] + cam.t[r];
            }
            float c[3][3];
            const float src[3][3] = {{su * eu[0], su * eu[1], su * eu[2]}, {sv * ev[0], sv * ev[1], sv * ev[2]},
                                     {pc[0], pc[1], pc[2]}};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                c[j][0] = cam.fx * src[j][0] + cam.cx * src[j][2];
                c[j][1] = cam.fy * src[j][1] + cam.cy * src[j][2];
                c[j][2] = src[j][2];
            }
            // adjugate rows a0 = c1 x c2, a1 = c2 x c0, a2 = c0 x c1;
            // d/dp (p x q).g = q x g, d/dq (p x q).g = g x p
            auto cross = [](const float* p, const float* q, float* o) {
                o[0] = p[1] * q[2] - p[2] * q[1];
                o[1] = p[2] * q[0] - p[0] * q[2];
                o[2] = p[0] * q[1] - p[1] * q[0];
            };
            float dc[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, tmp[3];
            cross(c[2], gA[0], tmp); for (int k = 0; k < 3; ++k) dc[1][k] += tmp[k];
            cross(gA[0], c[1], tmp); for (int k = 0; k < 3; ++k) dc[2][k] += tmp[k];
            cross(c[0], gA[1], tmp); for (int k = 0; k < 3; ++k) dc[2][k] += tmp[k];
            cross(gA[1], c[2], tmp); for (int k = 0; k < 3; ++k) dc[0][k] += tmp[k];
            cross(c[1], gA[2], tmp); for (int k = 0; k < 3; ++k) dc[0][k] += tmp[k];
            cross(gA[2], c[0], tmp); for (int k = 0; k < 3; ++k) dc[1][k] += tmp[k];
            // columns -> camera-space vectors (K^T), then world (Rv^T)
            float da[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                da[j][0] = cam.fx * dc[j][0];
                da[j][1] = cam.fy * dc[j][1];
                da[j][2] = cam.cx * dc[j][0] + cam.cy * dc[j][1] + dc[j][2];
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float rtu = cam.R[k] * da[0][0] + cam.R[3 + k] * da[0][1] + cam.R[6 + k] * da[0][2];
                const float rtv = cam.R[k] * da[1][0] + cam.R[3 + k] * da[1][1] + cam.R[6 + k] * da[1][2];
                gm[k] += cam.R[k] * da[2][0] + cam.R[3 + k] * da[2][1] + cam.R[6 + k] * da[2][2];
                dtu[k] += su * rtu;
                dtv[k] += sv * rtv;
            }
            gs[0] += eu[0] * da[0][0] + eu[1] * da[0][1] + eu[2] * da[0][2];
            gs[1] += ev[0] * da[1][0] + ev[1] * da[1][1] + ev[2] * da[1][2];
        }
        // t_u, t_v -> normalised quaternion -> raw quaternion
        const float Ju[4][3] = {{0, 2 * z, -2 * y}, {0, 2 * y, 2 * z}, {-4 * y, 2 * x, -2 * w}, {-4 * z, 2 * w, 2 * x}};
        const float Jv[4][3] = {{-2 * z, 0, 2 * x}, {2 * y, -4 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, -4 * z, 2 * y}};
        float dqh[4];
        const float qh[4] = {w, x, y, z};
        float dot = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dqh[k] = Ju[k][0] * dtu[0] + Ju[k][1] * dtu[1] + Ju[k][2] * dtu[2] + Jv[k][0] * dtv[0] +
                     Jv[k][1] * dtv[1] + Jv[k][2] * dtv[2];
            dot += dqh[k] * qh[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) gq[k] = (dqh[k] - dot * qh[k]) / qn;
    }
    if (a.g_means) { a.g_means[3 * s] = gm[0]; a.g_means[3 * s + 1] = gm[1]; a.g_means[3 * s + 2] = gm[2]; }
    if (a.g_scales) { a.g_scales[2 * s] = gs[0]; a.g_scales[2 * s + 1] = gs[1]; }
    if (a.g_quats) for (int k = 0; k < 4; ++k) a.g_quats[4 * s + k] = gq[k];
    if (a.g_opac) a.g_opac[s] = go;
    if (a.g_rgb) { a.g_rgb[3 * s] = gc[0]; a.g_rgb[3 * s + 1] = gc[1]; a.g_rgb[3 * s + 2] = gc[2]; }
}

// ---------------------------------------------------------------------------
// k_feat_out: g_feat[s] = slot >= 0 ? feat_acc[slot] : 0 (16-byte chunks)
// ---------------------------------------------------------------------------
template <typename FT>
__global__ void __launch_bounds__(256) k_feat_out(const __grid_constant__ RParams P, const BwdArgs a) {
    constexpr int E = FeatVec<FT>::E;
    const int nvec = P.C / E;
    const int64_t total = P.N * nvec;
    const bool err = a.st->err != 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / nvec;
        const int vv = (int)(i - s * nvec);
        const int slot = err ? -1 : a.splat_slot[s];
        float v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = 0.0f;
        if (slot >= 0) {
            const float4* src = reinterpret_cast<const float4*>(a.feat_acc + (int64_t)slot * P.C + vv * E);
#pragma unroll
            for (int k = 0; k < E / 4; ++k) {
                const float4 q = src[k];
                v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
            }
        }
        store_vec<E>(a.g_feat, s * P.C + vv * E, v, P.feat_dtype);
    }
}

// zero the gradient slots in use: grad rows (all views) and feature rows
__global__ void __launch_bounds__(256) k_bwd_clear(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                   const BwdArgs a) {
    const int64_t ns = a.st->nslot;
    const int64_t g4 = ns * (GRAD_STRIDE / 4);
    const int64_t f4 = ns * (P.C / 4);
    const int64_t total = g4 * cams.n + f4;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < g4 * cams.n) {
            const int64_t v = i / g4, r = i - v * g4;
            reinterpret_cast<float4*>(a.grad_item + v * P.N * GRAD_STRIDE)[r] = z;
        } else {
            reinterpret_cast<float4*>(a.feat_acc)[i - g4 * cams.n] = z;
        }
    }
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------
namespace {

cudaError_t set_smem(const void* k, size_t smem) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

template <typename FT>
cudaError_t launch_feat(const Cams& cams, const RParams& P, const BwdArgs& a, cudaStream_t s) {
    const size_t row = (size_t)P.C * 8;  // staged feature + accumulator, f32
    const size_t budget = 96 * 1024 - 2 * PCAP * 4;
    const int ucap = (int)std::max<size_t>(1, std::min<size_t>(1024, budget / row));
    const size_t smem = 2 * PCAP * 4 + (size_t)ucap * row;
    cudaError_t e;
#define FSS_FEAT(CPL)                                                                        \
    e = set_smem((const void*)k_bwd_feat<CPL, FT>, smem);                                  \
    if (e != cudaSuccess) return e;                                                         \
    k_bwd_feat<CPL, FT><<<cams.total_tiles, BWD_FEAT_THREADS, smem, s>>>(cams, P, a, ucap); \
    return cudaGetLastError();
    if (P.C <= 32) { FSS_FEAT(1) }
    if (P.C <= 64) { FSS_FEAT(2) }
    if (P.C <= 128) { FSS_FEAT(4) }
    if (P.C <= 256) { FSS_FEAT(8) }
    FSS_FEAT(16)
#undef FSS_FEAT
}

template <int TS, bool FULL, int CMAX, typename FT>
cudaError_t launch_geo_one(const Cams& cams, const RParams& P, const BwdArgs& a, cudaStream_t s) {
    constexpr int NB = FULL ? FBATCH : BB;
    const size_t smem = (size_t)NB * (3 * 16 + 4 * 4) + (size_t)NB * 16 * 4 + (FULL ? (size_t)NB * P.C * 8 : 0);
    cudaError_t e = set_smem((const void*)k_bwd_geo<TS, FULL, CMAX, FT>, smem);
    if (e != cudaSuccess) return e;
    k_bwd_geo<TS, FULL, CMAX, FT><<<cams.total_tiles, TS * TS, smem, s>>>(cams, P, a);
    return cudaGetLastError();
}

template <int TS, typename FT>
cudaError_t launch_geo(const Cams& cams, const RParams& P, const BwdArgs& a, cudaStream_t s) {
    if (P.K > 0) return launch_geo_one<TS, false, 4, FT>(cams, P, a, s);
    if (P.C <= 32) return launch_geo_one<TS, true, 32, FT>(cams, P, a, s);
    if (P.C <= 64) return launch_geo_one<TS, true, 64, FT>(cams, P, a, s);
    return launch_geo_one<TS, true, 128, FT>(cams, P, a, s);
}

template <typename FT>
cudaError_t launch_all(const Cams& cams, const RParams& P, const BwdArgs& a, int num_sms, cudaStream_t s) {
    cudaError_t e;
    k_bwd_clear<<<num_sms * 4, 256, 0, s>>>(cams, P, a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (P.K > 0) {
        if ((e = launch_feat<FT>(cams, P, a, s)) != cudaSuccess) return e;
    }
    if (P.ts == 8) e = launch_geo<8, FT>(cams, P, a, s);
    else if (P.ts == 16) e = launch_geo<16, FT>(cams, P, a, s);
    else e = launch_geo<32, FT>(cams, P, a, s);
    if (e != cudaSuccess) return e;
    const int64_t nb = (P.N + 255) / 256;
    k_bwd_project<<<(unsigned)std::max<int64_t>(1, nb), 256, 0, s>>>(cams, P, a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.g_feat) {
        k_feat_out<FT><<<num_sms * 8, 256, 0, s>>>(P, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_render_backward(const Cams& cams, const RParams& P, const BwdArgs& a, int num_sms,
                                   cudaStream_t stream) {
    if (P.feat_dtype == FSS_BF16) return launch_all<__nv_bfloat16>(cams, P, a, num_sms, stream);
    return launch_all<float>(cams, P, a, num_sms, stream);
}

}  // namespace fss
