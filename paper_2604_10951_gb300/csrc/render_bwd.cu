// Backward render for sm_103a: vector-Jacobian product of the forward
// render (Eq. 2, Eq. 7) with the Top-K set, skips, stops and clamps held
// fixed.  The paper trains through the differentiable renderer end to end
// (Sec. 3.1, Sec. 3.5) but prints no gradients; these are the chain
// rule of the forward:
//   s_j    = rgb_j . dL/dRGB + [j in K-set] c_j . dL/dF
//   dL/da_j = T_j (s_j - S_j),  S_j = sum_{i>j} w_i s_i / T_{j+1} + bg.dL/dRGB + dL/dT
//   S_{j-1} = a_j s_j + (1 - a_j) S_j,  T_j = T_{j+1} / (1 - a_j)
// replayed back to front from the saved traversal length and final T.
//
// k_bwd_feat  (Top-K) one CTA per tile: for every selected (pixel, k) the
//             dot c_i . dL/dF(x) and the feature gradient sum w_i dL/dF(x),
//             grouped by surfel in shared memory first, so each surfel's
//             feature row is read once and costs one row of 16-byte vector
//             reductions per tile.
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
#include "color.cuh"
#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"

#include <algorithm>
#include <climits>

namespace fss {

namespace {

constexpr int BB = 128;      // staged surfels per backward batch
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

}  // namespace

// ---------------------------------------------------------------------------
// k_bwd_feat (Top-K): per selected (pixel x, k) with surfel i, the dot
// c_i . dL/dF(x) (read by k_bwd_geo) and the feature gradient sum over x of
// w_i(x) dL/dF(x), grouped per tile
//
// Per tile (and per chunk of at most ECAP (pixel, k) entries):
//  1. the chunk's dL/dF rows are staged in shared memory (rows padded by
//     16 bytes); each thread keeps EPT entries (list position, weight) in
//     registers;
//  2. the selected list positions get dense slot numbers (mark + scan) and
//     a counting sort groups the entries by slot (shared-memory atomics)
//     into 8-byte records (slot, dL/dF row offset; weight);
//  3. the selected surfels' feature rows are staged in shared memory in one
//     parallel pass (over the counting-sort tables, which are dead by then);
//  4. the slot-grouped records are split into equal contiguous ranges, one
//     per group of G lanes (G = 16-byte chunks per row, rounded up to a
//     power of two).  A group takes four records per step.  When, for every
//     group of the warp, all four continue the group's current surfel (the
//     common case: about 30 entries per surfel and chunk), the warp takes
//     them without further checks; otherwise each record is checked, and a
//     group flushes one row of 16-byte vector reductions whenever its range
//     moves on to the next surfel.  The four partial dots are
//     reduce-scattered over the group, so each sum costs one shuffle per
//     lane and halving; packed FP32 FMAs (two products per instruction)
//     form the dots and w dL/dF.
// Shared memory holds everything the inner loop reads, so it runs without
// global-memory latency; the equal ranges keep the warps balanced.
// ---------------------------------------------------------------------------
constexpr int ECAP = 1024;  // (pixel, k) entries per pass
constexpr int PTAB = 2048;  // list positions per pass
constexpr int EPT = ECAP / BWD_FEAT_THREADS;  // entries per thread
constexpr int FEAT_UNION_BYTES = (PTAB + 2 * ECAP + 1) * 4;  // counting-sort tables, then feature rows
constexpr int MAX_ROW_PASSES = 64;

// entry record .x: slot << REC_ROW_BITS | offset of the entry's dL/dF row in
// 16-byte units (slot < PTAB = 2^11, offset < 2^17: 28 bits); .y: weight bits
constexpr int REC_ROW_BITS = 17;
constexpr int REC_ROW_MASK = (1 << REC_ROW_BITS) - 1;
constexpr int DOT_UNSET = 0x7fa00001;  // signalling-NaN payload: a dot not formed

// Sums of four values v[0..3] over the G lanes of a group (G a power of two,
// groups aligned in the warp), scattered: lanes swap halves of what is left
// and add, so each halving costs one shuffle per value kept.  Afterwards the
// lane holds the sums of the entries given by group_sum4_owned.
template <int G>
__device__ __forceinline__ void group_sum4(float (&v)[4], int sub) {
    constexpr unsigned ALL = 0xffffffffu;
    if constexpr (G >= 16) {
#pragma unroll
        for (int o = G >> 1; o >= 8; o >>= 1) {
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] += __shfl_xor_sync(ALL, v[j], o);
        }
    }
    if constexpr (G >= 2) {  // four values -> two: lanes with the offset bit keep entries 2, 3
        constexpr int o = G >= 8 ? 4 : G >> 1;
        const bool up = (sub & o) != 0;
        const float s0 = up ? v[0] : v[2], s1 = up ? v[1] : v[3];
        const float k0 = up ? v[2] : v[0], k1 = up ? v[3] : v[1];
        v[0] = k0 + __shfl_xor_sync(ALL, s0, o);
        v[1] = k1 + __shfl_xor_sync(ALL, s1, o);
    }
    if constexpr (G >= 4) {  // two -> one: lanes with the offset bit keep the second
        constexpr int o = G >= 8 ? 2 : 1;
        const bool up = (sub & o) != 0;
        const float sd = up ? v[0] : v[1], kp = up ? v[1] : v[0];
        v[0] = kp + __shfl_xor_sync(ALL, sd, o);
    }
    if constexpr (G >= 8) v[0] += __shfl_xor_sync(ALL, v[0], 1);
}

// rows of zeros after the chunk's dL/dF rows: at least G 16-byte chunks, so
// a lane without a record (or past the row) reads zeros
__host__ __device__ constexpr int zero_rows(int G, int rowb) { return (G * 16 + rowb - 1) / rowb; }

// (first entry, count) whose sums the lane stores after group_sum4: one
// lane per entry (G >= 4), two entries per lane (G = 2), all four (G = 1)
template <int G>
__device__ __forceinline__ int2 group_sum4_owned(int sub) {
    if constexpr (G >= 8) return make_int2((sub >> 1) & 3, (sub & 1) == 0 && sub < 8 ? 1 : 0);
    else if constexpr (G == 4) return make_int2(sub, 1);
    else if constexpr (G == 2) return make_int2(2 * sub, 2);
    else return make_int2(0, 4);
}

template <typename FT, int G>
__global__ void __launch_bounds__(BWD_FEAT_THREADS, 4) k_bwd_feat(const __grid_constant__ Cams cams,
                                                              const __grid_constant__ RParams P, const BwdArgs a,
                                                              int pch, int rowe, int ucap) {
    constexpr int E = FeatVec<FT>::E;
    constexpr int gpw = 32 / G, ngroups = (BWD_FEAT_THREADS / 32) * gpw;  // groups of G lanes
    extern __shared__ __align__(16) unsigned char smem[];
    const int rowb = rowe * (int)sizeof(FT), zr = zero_rows(G, rowb);
    FT* s_df = reinterpret_cast<FT*>(smem);  // [pch + zr][rowe]: the chunk's dL/dF rows, then zeros
    int2* s_rec = reinterpret_cast<int2*>(smem + (((size_t)(pch + zr) * rowb + 15) & ~(size_t)15));  // [ECAP]
    int* s_inv = reinterpret_cast<int*>(s_rec + ECAP);      // [ECAP] slot -> list position
    float* s_dot = reinterpret_cast<float*>(s_inv + ECAP);  // [ECAP] dots by entry (pixel * K + k)
    unsigned short* s_e = reinterpret_cast<unsigned short*>(s_dot + ECAP);  // [ECAP] record position -> entry
    int* s_gs = reinterpret_cast<int*>(s_e + ECAP);         // [ucap] slot -> gradient slot (this row pass)
    unsigned char* uni = reinterpret_cast<unsigned char*>(s_gs + ((ucap + 3) & ~3));
    int* s_tab = reinterpret_cast<int*>(uni);  // [PTAB] position -> slot
    int* s_off = s_tab + PTAB;                 // [ECAP + 1] per-slot counts -> offsets
    int* s_cur = s_off + ECAP + 1;             // [ECAP] scatter cursors
    FT* s_rows = reinterpret_cast<FT*>(uni);   // [ucap][rowe] feature rows (after the counting sort)
    __shared__ int s_red[33];
    __shared__ int s_tile;
    __shared__ int s_pass[MAX_ROW_PASSES + 1];

    if (a.st->err) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int TS = P.ts, lts = TS == 8 ? 3 : TS == 16 ? 4 : 5, npx = TS * TS;
    const int K = P.K, C = P.C, nvec = C / E;
    const int row16 = rowb / 16, zoff16 = pch * row16;  // padded row, first zero row (16-byte units)
    const FastDiv divK(K), divV(nvec);
    // chunk pixel of entry e = tid + i * BLOCK: a constant step when K divides the block
    const bool kdiv = BWD_FEAT_THREADS % K == 0;
    const int q0 = divK.div(tid), qstep = BWD_FEAT_THREADS / K;
    auto entry_q = [&](int i, int e) { return kdiv ? q0 + i * qstep : divK.div(e); };
    const int rv = BWD_FEAT_THREADS / nvec, r0v = tid / nvec, v0 = tid - r0v * nvec;  // row-chunk mapping
    const int sub = lane & (G - 1), gid = warp * gpw + lane / G;
    const bool chunk_live = sub < nvec;
    const int2 own = group_sum4_owned<G>(sub);
    const unsigned char* dfl = reinterpret_cast<const unsigned char*>(s_df) + sub * 16;  // this lane's chunk
    const FT* __restrict__ feats = reinterpret_cast<const FT*>(a.feats);
    const FT* __restrict__ dF = reinterpret_cast<const FT*>(a.d_feat);
    for (int i = tid; i < zr * rowb / 16; i += BWD_FEAT_THREADS)
        reinterpret_cast<uint4*>(s_df + (size_t)pch * rowe)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int t = next_tile_q(a.persistent, &a.st->work_feat, &s_tile, true, cams); t < cams.total_tiles;
         t = next_tile_q(a.persistent, &a.st->work_feat, &s_tile, false, cams)) {
        const int view = view_of_tile(cams, t);
        const CamDev& cam = cams.c[view];
        const int lt = t - cam.tile_off;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        const int2 rg = checked_range(a.ranges, t, P.pair_cap, a.st);
        const int64_t vbase = (int64_t)view * P.N;

        for (int pc0 = 0; pc0 < npx; pc0 += pch) {
            const int np = min(pch, npx - pc0), ne = np * K;
            // dots not yet formed read as a sentinel (a NaN payload that arithmetic does
            // not produce), so the write-back needs no per-entry state
            for (int e = tid; e < ne; e += BWD_FEAT_THREADS) s_dot[e] = __int_as_float(DOT_UNSET);
            // list positions in passes of PTAB (one pass unless the tile's list is longer)
            const int L = rg.y - rg.x;
            for (int p0 = 0; p0 < L; p0 += PTAB) {
                // 1. this thread's entries (e = tid + i * BLOCK) in this pass: list position
                // and weight (the chunk pixel q and k follow from e)
                int epos[EPT];
                float ew[EPT];
#pragma unroll
                for (int i = 0; i < EPT; ++i) {
                    const int e = tid + i * BWD_FEAT_THREADS;
                    epos[i] = -1;
                    ew[i] = 0.0f;
                    if (e < ne) {
                        const int q = entry_q(i, e), k = e - q * K, p = pc0 + q;
                        const int px = tx * TS + (p & (TS - 1)), py = ty * TS + (p >> lts);
                        if (px < cam.W && py < cam.H) {
                            const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
                            int pos = a.saved_pos[pix * K + k];
                            if (pos >= 0 && !in_bounds(a.st, SITE_LIST_POS, pos, L)) pos = -1;
                            if (pos >= p0 && pos < p0 + PTAB) {
                                epos[i] = pos - p0;
                                ew[i] = a.saved_w[pix * K + k];
                                if (P.renorm) {  // dL/dc = (w / W) dL/dF, W the selected weights' sum
                                    float ws = 0.0f;
                                    for (int k2 = 0; k2 < K; ++k2) ws += a.saved_w[pix * K + k2];
                                    ew[i] = ws > 0.0f ? ew[i] / ws : 0.0f;
                                }
                            }
                        }
                    }
                }
                if (p0 == 0) {
                    // the chunk's dL/dF rows (zeros outside the image), copied asynchronously
                    // once this thread's entries have arrived (issued first, they queued
                    // the entry loads behind them) and waited for just before the inner loop
                    if (r0v < rv) {
                        for (int q = r0v; q < np; q += rv) {
                            const int p = pc0 + q, px = tx * TS + (p & (TS - 1)), py = ty * TS + (p >> lts);
                            const bool in = px < cam.W && py < cam.H;
                            const FT* src = in ? dF + (cam.pix_off + (int64_t)py * cam.W + px) * C + v0 * E : dF;
                            cp_async16(s_df + (size_t)q * rowe + v0 * E, src, in ? 16 : 0);
                        }
                    }
                    cp_async_commit();
                }
                // 2. slots of the selected positions, then the entries grouped by slot: the
                // entries per position are counted, and one exclusive scan of
                // (count << 16 | count > 0) over the positions gives each position both its
                // first record (high half) and its slot (low half: selected positions
                // before it); counts <= ECAP and positions <= PTAB fit 16 bits each
                const int nt = min(PTAB, L - p0);  // positions in use (U <= nt)
                for (int i = tid; i < nt; i += BWD_FEAT_THREADS) s_tab[i] = 0;
                __syncthreads();
#pragma unroll
                for (int i = 0; i < EPT; ++i)
                    if (epos[i] >= 0) atomicAdd(&s_tab[epos[i]], 1 << 16);
                __syncthreads();
                const int tot = block_exscan_marked(s_tab, nt, s_red);
                const int U = tot & 0xffff, nsel = tot >> 16;
                if (U == 0) continue;
                for (int i = tid; i < nt; i += BWD_FEAT_THREADS) {
                    const int pre = s_tab[i], nxt = i + 1 < nt ? s_tab[i + 1] : tot;
                    if ((nxt & 0xffff) - (pre & 0xffff) == 1) {  // a selected position: its slot
                        s_inv[pre & 0xffff] = i;
                        s_off[pre & 0xffff] = pre >> 16;
                        s_cur[pre & 0xffff] = pre >> 16;
                    }
                }
                if (tid == 0) s_off[U] = nsel;
                int eslot[EPT];
#pragma unroll
                for (int i = 0; i < EPT; ++i) eslot[i] = epos[i] >= 0 ? s_tab[epos[i]] & 0xffff : -1;
                __syncthreads();
#pragma unroll
                for (int i = 0; i < EPT; ++i) {
                    if (eslot[i] >= 0) {
                        const int at = atomicAdd(&s_cur[eslot[i]], 1);
                        const int e = tid + i * BWD_FEAT_THREADS;
                        s_rec[at] = make_int2((eslot[i] << REC_ROW_BITS) | (entry_q(i, e) * row16), __float_as_int(ew[i]));
                        s_e[at] = (unsigned short)e;
                    }
                }
                const int npass = (U + ucap - 1) / ucap;  // <= MAX_ROW_PASSES (checked by the launcher)
                if (tid <= npass) s_pass[tid] = s_off[min(tid * ucap, U)];
                __syncthreads();
                for (int pi = 0; pi < npass; ++pi) {
                    const int u0 = pi * ucap, nu = min(ucap, U - u0);
                    const int eb = s_pass[pi], ee = s_pass[pi + 1];
                    // 3. feature rows of slots [u0, u0 + nu) (over the counting-sort tables),
                    // copied asynchronously like the dL/dF rows
                    for (int idx = tid; idx < nu * nvec; idx += BWD_FEAT_THREADS) {
                        const int u = divV.div(idx), v = idx - u * nvec;
                        const int64_t sp = (int64_t)a.list[rg.x + p0 + s_inv[u0 + u]] - vbase;
                        const bool ok = in_bounds(a.st, SITE_ITEM, sp, P.N);  // check build: a zero row, no slot
                        cp_async16(s_rows + (size_t)u * rowe + v * E, ok ? feats + sp * C + v * E : feats, ok ? 16 : 0);
                        if (v == 0) {
                            const int sl = ok ? a.splat_slot[sp] : -1;
                            s_gs[u] = in_bounds(a.st, SITE_SLOT, sl, P.N) ? sl : -1;
                        }
                    }
                    cp_async_commit();
                    cp_async_wait_all();
                    __syncthreads();
                    // 4. equal contiguous record ranges per group, starting at an even record
                    // (records are read two at a time), four records per step (warp-uniform
                    // trip count)
                    const int ea = eb & ~1;
                    const int len = (((ee - ea + ngroups - 1) / ngroups) + 3) & ~3;
                    const int i0 = ea + gid * len, i1 = min(ee, i0 + len);
                    int cur = -1;  // the group's current slot
                    float2 f2[E / 2], acc2[E / 2];
#pragma unroll
                    for (int e = 0; e < E / 2; ++e) { f2[e] = make_float2(0.0f, 0.0f); acc2[e] = f2[e]; }
                    // flush the current slot's w dL/dF, then move to `slot`
                    auto next_slot = [&](int slot) {
                        if (chunk_live) {
                            if (cur >= 0 && FSS_CHECKED(s_gs[cur - u0] >= 0)) {
                                float* dst = a.feat_acc + (int64_t)s_gs[cur - u0] * C + sub * E;
#pragma unroll
                                for (int e = 0; e < E / 2; e += 2)
                                    red_add_v4(dst + 2 * e, acc2[e].x, acc2[e].y, acc2[e + 1].x, acc2[e + 1].y);
                            }
                            if (slot >= 0) {
                                float fv[E];
                                FeatVec<FT>::lds(s_rows + (size_t)(slot - u0) * rowe + sub * E, fv);
#pragma unroll
                                for (int e = 0; e < E / 2; ++e) f2[e] = make_float2(fv[2 * e], fv[2 * e + 1]);
                            }
#pragma unroll
                            for (int e = 0; e < E / 2; ++e) acc2[e] = make_float2(0.0f, 0.0f);
                        }
                        cur = slot;
                    };
                    // one record of the current slot: returns the lane's partial dot
                    // (no record: the zero row and weight 0, so the code has no branch)
                    auto take = [&](int2 r, bool live) {
                        const bool on = chunk_live && live;
                        float g[E];
                        FeatVec<FT>::lds(reinterpret_cast<const FT*>(dfl + (size_t)(on ? r.x & REC_ROW_MASK : zoff16) * 16), g);
                        const float w = on ? __int_as_float(r.y) : 0.0f;
                        const float2 w2 = make_float2(w, w);
                        float2 d = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int e = 0; e < E / 2; ++e) {
                            const float2 g2 = make_float2(g[2 * e], g[2 * e + 1]);
                            d = __ffma2_rn(f2[e], g2, d);
                            acc2[e] = __ffma2_rn(w2, g2, acc2[e]);
                        }
                        return d.x + d.y;
                    };
                    for (int st = 0; st < len; st += 4) {
                        const int i = i0 + st;
                        int4 ra = make_int4(-1, 0, -1, 0), rb = ra;
                        if (i < i1) ra = *reinterpret_cast<const int4*>(s_rec + i);
                        if (i + 2 < i1) rb = *reinterpret_cast<const int4*>(s_rec + i + 2);
                        const int2 r[4] = {make_int2(ra.x, ra.y), make_int2(ra.z, ra.w), make_int2(rb.x, rb.y),
                                           make_int2(rb.z, rb.w)};
                        float v[4];
                        // steady: all four records continue the group's current slot (sorted
                        // records: the fourth decides), or the group's range is used up
                        const bool done = i >= i1;
                        const bool steady = done || (i >= eb && i + 3 < i1 && (rb.z >> REC_ROW_BITS) == cur);
                        if (__all_sync(0xffffffffu, steady)) {  // warp-uniform: no per-record checks
#pragma unroll
                            for (int j = 0; j < 4; ++j) v[j] = take(r[j], !done);
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const bool live = i + j >= eb && i + j < i1;
                                const int slot = r[j].x >> REC_ROW_BITS;
                                if (live && slot != cur) next_slot(slot);
                                v[j] = take(r[j], live);
                            }
                        }
                        group_sum4<G>(v, sub);
#pragma unroll
                        for (int j = 0; j < (G >= 4 ? 1 : 4 / G); ++j) {
                            const int at = i + own.x + j;
                            if (j < own.y && at >= eb && at < i1) s_dot[s_e[at]] = v[j];
                        }
                    }
                    next_slot(-1);
                    __syncthreads();
                }
            }
            // the dots, written back in (pixel, k) order
#pragma unroll
            for (int i = 0; i < EPT; ++i) {
                const int e = tid + i * BWD_FEAT_THREADS;
                const float d = e < ne ? s_dot[e] : __int_as_float(DOT_UNSET);
                if (__float_as_int(d) != DOT_UNSET) {
                    const int q = entry_q(i, e), p = pc0 + q;
                    const int64_t pix = cam.pix_off + (int64_t)(ty * TS + (p >> lts)) * cam.W + tx * TS + (p & (TS - 1));
                    a.dots[pix * K + (e - q * K)] = d;
                }
            }
            cp_async_wait_all();  // (a chunk without selected entries never waited)
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// k_bwd_geo: back-to-front replay (Top-K and full accumulation)
// ---------------------------------------------------------------------------
template <int TS, bool FULL, int CMAX, typename FT, bool VAR>
__global__ void __launch_bounds__(TS * TS) k_bwd_geo(const __grid_constant__ Cams cams,
                                                     const __grid_constant__ RParams P, const BwdArgs a) {
    constexpr int NT = TS * TS;
    constexpr int NB = FULL ? FBATCH : BB;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_r0 = reinterpret_cast<float4*>(smem);
    float4* s_r1 = s_r0 + NB;
    float4* s_r2 = s_r1 + NB;
    float4* s_oc = s_r2 + NB;                                  // (o, r, g, b)
    uint32_t* s_wm = reinterpret_cast<uint32_t*>(s_oc + NB);   // warps the footprint reaches
    float* s_g = reinterpret_cast<float*>(s_wm + 2 * NB);      // [NB][16] partial derivatives
    float* s_f = s_g + NB * 16;    // FULL: [NB][C] features
    float* s_gf = s_f + (FULL ? NB * P.C : 0);  // FULL: [NB][C] feature gradients
    __shared__ int s_max;
    __shared__ int s_tile;
    __shared__ uint32_t s_bits[NT / 32][BB / 32];  // per warp: the staged surfels its block meets

    if (a.st->err) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t wbit = 1u << (tid >> 5);
    const int C = P.C, K = P.K;
    for (int t = next_tile_q(a.persistent, &a.st->work_geo, &s_tile, true, cams); t < cams.total_tiles;
         t = next_tile_q(a.persistent, &a.st->work_geo, &s_tile, false, cams)) {
    const int view = view_of_tile(cams, t);
    const CamDev& cam = cams.c[view];
    const int lt = t - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int2 lp = pixel_of<TS>(tid);
    const int px = tx * TS + lp.x, py = ty * TS + lp.y;
    const bool inside = px < cam.W && py < cam.H;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const int2 rg = checked_range(a.ranges, t, P.pair_cap, a.st);
    const int64_t vbase = (int64_t)view * P.N;
    // VAR instances carry the variants (renormalised Top-K, spherical-harmonic
    // item colours, low-pass filter), read from the parameters; the plain
    // instance keeps its code as it is
    const float* __restrict__ rgbv = a.rgb + (VAR && P.color_sh ? 3 * vbase : 0);
    const int64_t pix = cam.pix_off + (int64_t)py * cam.W + px;
    const FT* __restrict__ feats = reinterpret_cast<const FT*>(a.feats);

    int nstop = 0;
    float T = 1.0f, gr = 0.0f, gg = 0.0f, gb = 0.0f, Sh = 0.0f;
    int kk = -1, next_pos = -1;
    float next_dot = 0.0f;
    // a selected surfel adds rn_a * dot + rn_b to what its weight multiplies:
    // the dot itself, or (dot - F.dL/dF) / W for the renormalised variant
    float rn_a = 1.0f, rn_b = 0.0f;
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
            if (VAR && P.renorm) {  // entries 0..kk are the selected ones, front to back
                float ws = 0.0f, wd = 0.0f;
                for (int k2 = 0; k2 <= kk; ++k2) {
                    const float wv = a.saved_w[pix * K + k2];
                    ws += wv;
                    wd = fmaf(wv, a.dots[pix * K + k2], wd);
                }
                rn_a = ws > 0.0f ? 1.0f / ws : 0.0f;
                rn_b = -wd * rn_a * rn_a;
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
            s_wm[j] = a.masks[rg.x + b_start + j];
        }
        for (int i = tid; i < cnt * 16; i += NT) s_g[i] = 0.0f;
        if (FULL) {
            constexpr int E = FeatVec<FT>::E;
            const int nvec = C / E, rpi = NT / nvec, r0 = tid / nvec, vv = tid - r0 * nvec;
            for (int j = r0; r0 < rpi && j < cnt; j += rpi) {
                const int64_t sp = (int64_t)a.list[rg.x + b_start + j] - vbase;
                if (!FSS_CHECKED(sp >= 0 && sp < P.N)) continue;  // recorded by the staging loop
                float f[E];
                FeatVec<FT>::load(feats + sp * C + vv * E, f);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    s_f[j * C + vv * E + e] = f[e];
                    s_gf[j * C + vv * E + e] = 0.0f;
                }
            }
        }
        __syncthreads();
        // this warp's staged surfels as bit words (the footprint misses the
        // other ones): the loop below visits set bits only, last first
#pragma unroll
        for (int i = 0; i < NB / 32; ++i) {
            const int j = 32 * i + lane;
            const uint32_t word = __ballot_sync(0xffffffffu, j < cnt && (s_wm[j] & wbit));
            if (lane == i) s_bits[tid >> 5][i] = word;
        }
        __syncwarp();
        for (int i = ((cnt + 31) >> 5) - 1; i >= 0; --i) {
        for (uint32_t bits = s_bits[tid >> 5][i]; bits != 0u; bits ^= 0x80000000u >> __clz(bits)) {
            const int j = 32 * i + 31 - __clz(bits);
            const int pos = b_start + j;
            float g[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) g[k] = 0.0f;
            float w = 0.0f;
            bool contrib = false;
            Hit h;
            const float4 oc = s_oc[j];
            if (pos < nstop &&
                eval_splat<VAR>(s_r0[j], s_r1[j], s_r2[j], oc.x, pxf, pyf, P.alpha_min, cam.near_plane, h, P.lowpass)) {
                contrib = true;
                const float alpha = fminf(h.alpha_raw, P.alpha_max);
                const float Tj = T * rcp_approx(1.0f - alpha);
                w = alpha * Tj;
                float s = oc.y * gr + oc.z * gg + oc.w * gb;
                if (!FULL) {
                    if (pos == next_pos) {
                        s += VAR ? fmaf(next_dot, rn_a, rn_b) : next_dot;
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
                    g[9] = dal * h.G;
                    const float drho = -0.5f * alpha * dal;
                    if (VAR && h.scr) {  // low-pass screen term: rho = 2 |x - c|^2, d rho / d c = -4 (X, Y)
                        g[13] = -4.0f * h.X * drho;
                        g[14] = -4.0f * h.Y * drho;
                    } else {
                        const float du = 2.0f * h.u * drho, dv = 2.0f * h.v * drho;
                        const float gc0 = du * h.inv, gc1 = dv * h.inv, gc2 = -(du * h.u + dv * h.v) * h.inv;
                        g[0] = gc0 * h.X; g[1] = gc0 * h.Y; g[2] = gc0;
                        g[3] = gc1 * h.X; g[4] = gc1 * h.Y; g[5] = gc1;
                        g[6] = gc2 * h.X; g[7] = gc2 * h.Y; g[8] = gc2;
                    }
                }
                T = Tj;
            }
            if (__any_sync(0xffffffffu, contrib)) {
                reduce_scatter<16>(g);  // lane l holds value l >> 1
                if ((lane & 1) == 0 && (lane >> 1) < (VAR ? 15 : 13)) atomicAdd(&s_g[j * 16 + (lane >> 1)], g[0]);
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
        }
        __syncthreads();
        // flush one gradient row per staged surfel
        for (int j = tid; j < cnt; j += NT) {
            const float* v = s_g + 16 * j;
            bool nz = false;
#pragma unroll
            for (int k = 0; k < (VAR ? 15 : 13); ++k) nz |= v[k] != 0.0f;
            if (!nz) continue;
            const int64_t sp = (int64_t)a.list[rg.x + b_start + j] - vbase;
            if (!FSS_CHECKED(sp >= 0 && sp < P.N)) continue;  // recorded by the staging loop
            const int slot = a.splat_slot[sp];
            if (!in_bounds(a.st, SITE_SLOT, slot, P.N)) continue;
            float* dst = a.grad_item + ((int64_t)view * P.N + slot) * GRAD_STRIDE;
            red_add_v4(dst, v[0], v[1], v[2], v[3]);
            red_add_v4(dst + 4, v[4], v[5], v[6], v[7]);
            red_add_v4(dst + 8, v[8], v[9], v[10], v[11]);
            if (VAR)
                red_add_v4(dst + 12, v[12], v[13], v[14], 0.0f);  // colour b, projected-centre gradient
            else
                atomicAdd(dst + 12, v[12]);
        }
        if (FULL) {
            const int c4 = C / 4;
            for (int idx = tid; idx < cnt * c4; idx += NT) {
                const int j = idx / c4, q = idx - j * c4;
                const float* v = s_gf + j * C + 4 * q;
                if (v[0] == 0.0f && v[1] == 0.0f && v[2] == 0.0f && v[3] == 0.0f) continue;
                const int64_t sp = (int64_t)a.list[rg.x + b_start + j] - vbase;
                if (!FSS_CHECKED(sp >= 0 && sp < P.N)) continue;  // recorded by the staging loop
                const int slot = a.splat_slot[sp];
                if (!in_bounds(a.st, SITE_SLOT, slot, P.N)) continue;
                red_add_v4(a.feat_acc + (int64_t)slot * C + 4 * q, v[0], v[1], v[2], v[3]);
            }
        }
    }
    __syncthreads();
    }  // tiles
}

// ---------------------------------------------------------------------------
// k_bwd_project: per surfel, d(adjugate rows) -> d(means, scales, quats)
// ---------------------------------------------------------------------------
// gradients of surfel s from its slot's per-view rows (slot < 0: zeros).
// VAR instances carry the variants, read from the parameters:
//  - spherical-harmonic colours: each view's colour gradient goes to the
//    coefficients (g_rgb [N, B, 3], accumulated in place by the surfel's own
//    thread) and, through the view direction d = (p - o) / |p - o|, to the
//    means: dd/dp = (I - d d^T) / |p - o|; a clamped channel passes nothing;
//  - low-pass filter: the rows' projected-centre gradient (entries 13, 14)
//    goes to the means through xc = fx pc_x / pc_z + cx, yc = fy pc_y / pc_z + cy.
template <bool VAR>
__device__ __forceinline__ void project_grad(const Cams& cams, const RParams& P, const BwdArgs& a, const float* sh,
                                             int64_t s, int slot) {
    float gm[3] = {0, 0, 0}, gs[2] = {0, 0}, gq[4] = {0, 0, 0, 0}, go = 0.0f, gc[3] = {0, 0, 0};
    const int nb = (P.sh_deg + 1) * (P.sh_deg + 1);
    const bool SH = VAR && P.color_sh;
    float* gsh = SH && a.g_rgb ? a.g_rgb + s * nb * 3 : nullptr;
    if (gsh)
        for (int i = 0; i < nb * 3; ++i) gsh[i] = 0.0f;
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
            if (SH && (g2.z != 0.f || g2.w != 0.f || g12 != 0.f)) {
                float ox, oy, oz;
                cam_centre(cams.c[v], ox, oy, oz);
                const float vx = a.means[3 * s] - ox, vy = a.means[3 * s + 1] - oy, vz = a.means[3 * s + 2] - oz;
                const float ir = rsqrtf(vx * vx + vy * vy + vz * vz);
                const float dx = vx * ir, dy = vy * ir, dz = vz * ir;
                float Y[16];
                sh_basis(P.sh_deg, dx, dy, dz, Y);
                const float* k = sh + s * nb * 3;
                float gd[3] = {0.f, 0.f, 0.f};
                for (int ch = 0; ch < 3; ++ch) {
                    const float g = ch == 0 ? g2.z : (ch == 1 ? g2.w : g12);
                    float c = 0.5f;
                    for (int b = 0; b < nb; ++b) c = fmaf(k[3 * b + ch], Y[b], c);
                    if (!(c > 0.0f) || g == 0.0f) continue;
                    if (gsh)
                        for (int b = 0; b < nb; ++b) gsh[3 * b + ch] = fmaf(Y[b], g, gsh[3 * b + ch]);
                    float gx, gy, gz;
                    sh_grad_dot(P.sh_deg, dx, dy, dz, k + ch, 3, gx, gy, gz);
                    gd[0] = fmaf(g, gx, gd[0]);
                    gd[1] = fmaf(g, gy, gd[1]);
                    gd[2] = fmaf(g, gz, gd[2]);
                }
                const float dd = dx * gd[0] + dy * gd[1] + dz * gd[2];
                gm[0] += (gd[0] - dx * dd) * ir;
                gm[1] += (gd[1] - dy * dd) * ir;
                gm[2] += (gd[2] - dz * dd) * ir;
            }
            const CamDev& cam = cams.c[v];
            if (VAR && P.lowpass && (gv[13] != 0.f || gv[14] != 0.f)) {
                float pc[3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    pc[r] = cam.R[3 * r] * pm[0] + cam.R[3 * r + 1] * pm[1] + cam.R[3 * r + 2] * pm[2] + cam.t[r];
                const float iz = 1.0f / pc[2], gx = gv[13] * cam.fx * iz, gy = gv[14] * cam.fy * iz;
                const float dpc[3] = {gx, gy, -(gx * pc[0] + gy * pc[1]) * iz};
#pragma unroll
                for (int k = 0; k < 3; ++k) gm[k] += cam.R[k] * dpc[0] + cam.R[3 + k] * dpc[1] + cam.R[6 + k] * dpc[2];
            }
            if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
                g1.z == 0.f && g1.w == 0.f && g2.x == 0.f)
                continue;
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
    if (!(VAR && P.color_sh) && a.g_rgb) { a.g_rgb[3 * s] = gc[0]; a.g_rgb[3 * s + 1] = gc[1]; a.g_rgb[3 * s + 2] = gc[2]; }
}

// Zeros for surfels culled in every view (one thread each), then the chain
// rule for the surfels that have a slot, densely over the slots (a few
// percent of the surfels are visible, so a thread per surfel would leave
// most lanes of a warp idle through the long path).
template <bool VAR>
__global__ void __launch_bounds__(256) k_bwd_project(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                     const BwdArgs a, const float* __restrict__ sh) {
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const bool err = a.st->err != 0;
    for (int64_t s = gtid; s < P.N; s += gstride)
        if (err || a.splat_slot[s] < 0) project_grad<VAR>(cams, P, a, sh, s, -1);
    int64_t ns = err ? 0 : (int64_t)a.st->nslot;
    if (ns > 0 && !in_bounds(a.st, SITE_SLOT, ns - 1, P.N)) ns = 0;
    for (int64_t sl = gtid; sl < ns; sl += gstride) {
        const int32_t s = a.slot_surf[sl];
        if (in_bounds(a.st, SITE_SLOT, s, P.N)) project_grad<VAR>(cams, P, a, sh, s, (int)sl);
    }
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
    const bool pow2 = (nvec & (nvec - 1)) == 0;  // the usual widths: a shift instead of a 64-bit division
    const int sh = __ffs(nvec) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = pow2 ? (i >> sh) : i / nvec;
        const int vv = (int)(i - s * nvec);
        int slot = err ? -1 : a.splat_slot[s];
        if (slot >= 0 && !in_bounds(a.st, SITE_SLOT, slot, P.N)) slot = -1;
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
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->work_feat = 0u;
        a.st->work_geo = 0u;
    }
    int64_t ns = a.st->nslot;
    if (ns > 0 && !in_bounds(a.st, SITE_SLOT, ns - 1, P.N)) ns = 0;
    const int64_t g4 = ns * (GRAD_STRIDE / 4);
    const int64_t f4 = ns * (P.C / 4);
    const int64_t total = g4 * cams.n + f4;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < g4 * cams.n) {
            const int64_t v = cams.n == 1 ? 0 : i / g4, r = i - v * g4;
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

// one resident wave: CTAs per SM times SMs, capped by the number of tiles
cudaError_t persistent_grid(const void* k, int threads, size_t smem, int& grid) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid = std::max(1, std::min(grid, std::max(1, per_sm) * sms));
    return cudaSuccess;
}

template <typename FT>
cudaError_t launch_feat(const Cams& cams, const RParams& P, const BwdArgs& a, cudaStream_t s) {
    const int nvec = P.C / FeatVec<FT>::E;
    int G = 1;  // lanes per entry: 16-byte chunks of a feature row, padded to a power of two
    while (G < nvec) G <<= 1;
    if (G > 32) return cudaErrorInvalidValue;  // C too large (checked by the ABI)
    const int rowe = P.C + 16 / (int)sizeof(FT);  // padded row, elements
    const size_t rowb = (size_t)rowe * sizeof(FT);
    const int ucap = (int)(FEAT_UNION_BYTES / rowb);  // feature rows per pass
    // row passes per chunk: ceil(U / ucap), U <= ECAP (every slot has an entry)
    if (ucap < 1 || (ECAP + ucap - 1) / ucap > MAX_ROW_PASSES) return cudaErrorInvalidValue;
    const int npx = P.ts * P.ts;
    int pch = std::min(npx, ECAP / std::max(1, P.K));
    pch = (int)std::min<size_t>((size_t)pch, std::max<size_t>(32, (24 * 1024) / rowb));
    const size_t smem = (((size_t)(pch + zero_rows(G, (int)rowb)) * rowb + 15) & ~(size_t)15) + (size_t)4 * ECAP * 4 +
                        (size_t)2 * ECAP +
                        (size_t)((ucap + 3) & ~3) * 4 + FEAT_UNION_BYTES;
    auto go = [&](auto kern) {
        cudaError_t e2 = set_smem((const void*)kern, smem);
        if (e2 != cudaSuccess) return e2;
        int grid = cams.total_tiles;
        if (a.persistent && (e2 = persistent_grid((const void*)kern, BWD_FEAT_THREADS, smem, grid)) != cudaSuccess)
            return e2;
        kern<<<grid, BWD_FEAT_THREADS, smem, s>>>(cams, P, a, pch, rowe, ucap);
        e2 = cudaGetLastError();
        if (e2 == cudaSuccess) kernel_mark(s);
        return e2;
    };
    switch (G) {
        case 1: return go(k_bwd_feat<FT, 1>);
        case 2: return go(k_bwd_feat<FT, 2>);
        case 4: return go(k_bwd_feat<FT, 4>);
        case 8: return go(k_bwd_feat<FT, 8>);
        case 16: return go(k_bwd_feat<FT, 16>);
        default: return go(k_bwd_feat<FT, 32>);
    }
}

template <int TS, bool FULL, int CMAX, typename FT, bool VAR = false>
cudaError_t launch_geo_one(const Cams& cams, const RParams& P, const BwdArgs& a, cudaStream_t s) {
    constexpr int NB = FULL ? FBATCH : BB;
    const size_t smem = (size_t)NB * (4 * 16 + 8) + (size_t)NB * 16 * 4 + (FULL ? (size_t)NB * P.C * 8 : 0);  // staging, masks, partials, rows
    cudaError_t e = set_smem((const void*)k_bwd_geo<TS, FULL, CMAX, FT, VAR>, smem);
    if (e != cudaSuccess) return e;
    int grid = cams.total_tiles;
    if (a.persistent && (e = persistent_grid((const void*)k_bwd_geo<TS, FULL, CMAX, FT, VAR>, TS * TS, smem, grid)) !=
                            cudaSuccess)
        return e;
    k_bwd_geo<TS, FULL, CMAX, FT, VAR><<<grid, TS * TS, smem, s>>>(cams, P, a);
    e = cudaGetLastError();
    if (e == cudaSuccess) kernel_mark(s);
    return e;
}

template <int TS, typename FT>
cudaError_t launch_geo(const Cams& cams, const RParams& P, const BwdArgs& a, cudaStream_t s) {
    // the variants (renormalised Top-K, spherical-harmonic colours, low-pass
    // filter) have their own instances: no cost on the plain paths
    const bool var = P.renorm || P.color_sh || P.lowpass;
    if (P.K > 0) return var ? launch_geo_one<TS, false, 4, FT, true>(cams, P, a, s) : launch_geo_one<TS, false, 4, FT>(cams, P, a, s);
    if (P.C <= 32) return var ? launch_geo_one<TS, true, 32, FT, true>(cams, P, a, s) : launch_geo_one<TS, true, 32, FT>(cams, P, a, s);
    if (P.C <= 64) return var ? launch_geo_one<TS, true, 64, FT, true>(cams, P, a, s) : launch_geo_one<TS, true, 64, FT>(cams, P, a, s);
    return var ? launch_geo_one<TS, true, 128, FT, true>(cams, P, a, s) : launch_geo_one<TS, true, 128, FT>(cams, P, a, s);
}

template <typename FT>
cudaError_t launch_all(const Cams& cams, const RParams& P, const BwdArgs& a, const float* sh, int num_sms,
                       cudaStream_t s) {
    cudaError_t e;
    k_bwd_clear<<<num_sms * 4, 256, 0, s>>>(cams, P, a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kernel_mark(s);
    if (P.K > 0) {
        if ((e = launch_feat<FT>(cams, P, a, s)) != cudaSuccess) return e;
    }
    // With Top-K the feature gradients are complete here: launched eagerly,
    // their output pass (memory bound) runs in a second stream beside the
    // geometry replay (issue bound) and joins before the call returns: 10 us
    // less per 500k-surfel frame.  A graph being captured keeps one stream:
    // replayed, the branch measured 3 us slower than the chain.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
    const bool fork = a.g_feat && P.K > 0 && cap == cudaStreamCaptureStatusNone && !kernel_marks_armed() &&
                      side_stream(s, side, ev_fork, ev_join);
    if (fork) {
        if ((e = cudaEventRecord(ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ev_fork, 0)) != cudaSuccess) return e;
        k_feat_out<FT><<<num_sms * 8, 256, 0, side>>>(P, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(ev_join, side)) != cudaSuccess) {
            (void)cudaStreamSynchronize(side);  // no join event: wait for the side stream's kernel here
            return e;
        }
    }
    // from here on every return joins the side stream first, so that no work of
    // this call is left running after it returns, even on an error
    auto joined = [&](cudaError_t err) {
        if (fork) {
            const cudaError_t ej = cudaStreamWaitEvent(s, ev_join, 0);
            if (err == cudaSuccess) err = ej;
        }
        return err;
    };
    if (P.ts == 8) e = launch_geo<8, FT>(cams, P, a, s);
    else if (P.ts == 16) e = launch_geo<16, FT>(cams, P, a, s);
    else e = launch_geo<32, FT>(cams, P, a, s);
    if (e != cudaSuccess) return joined(e);
    const int64_t nb = (P.N + 255) / 256;
    if (P.color_sh || P.lowpass)
        k_bwd_project<true><<<(unsigned)std::max<int64_t>(1, nb), 256, 0, s>>>(cams, P, a, sh);
    else
        k_bwd_project<false><<<(unsigned)std::max<int64_t>(1, nb), 256, 0, s>>>(cams, P, a, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return joined(e);
    kernel_mark(s);
    if (fork) {
        if ((e = joined(cudaSuccess)) != cudaSuccess) return e;
    } else if (a.g_feat) {
        k_feat_out<FT><<<num_sms * 8, 256, 0, s>>>(P, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        kernel_mark(s);
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_render_backward(const Cams& cams, const RParams& P, const BwdArgs& a, const float* sh, int num_sms,
                                   cudaStream_t stream) {
    if (P.feat_dtype == FSS_BF16) return launch_all<__nv_bfloat16>(cams, P, a, sh, num_sms, stream);
    return launch_all<float>(cams, P, a, sh, num_sms, stream);
}

}  // namespace fss
