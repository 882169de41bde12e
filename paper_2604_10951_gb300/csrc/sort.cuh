// Per-tile depth sort (the paper composites the surfels in depth order,
// Sec. 3.1), as a CTA-wide device function: the sort kernel runs it with one
// CTA per tile, and the Top-K forward's SORT instances run it on their own
// tile before rendering it.
//
// Binning leaves every tile's range of the pair list filled in arbitrary
// order (bounded items first, then the view's unbounded items are appended
// here).  The CTA sorts its range by the 64-bit key
//   (binary32 bits of the item's camera depth) << 32 | item index,
// which is unique, so the order is total and deterministic.  Depths are
// positive, so their bit patterns order like the numbers.
//   - up to SORT_CAP keys: 32-key chunks sorted by one warp each in
//     registers, then merged by rank (place in the chunk plus a binary
//     search in every other chunk);
//   - longer lists: stable LSD radix sort (8-bit digits) by the same CTA
//     in a global scratch range of the same offsets.
// With the sorted item, each pair gets the mask of the tile's warps (8 x 4
// pixel blocks) that its footprint reaches, which the render passes use
// to skip a surfel warp by warp.
#pragma once

#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"

namespace fss {

// shared memory of sort_tile: keys, masks (by list position), positions
constexpr size_t SORT_SMEM_BYTES = (size_t)SORT_CAP * (8 + 4 + 2);

namespace {

__device__ __forceinline__ uint64_t sort_key(const float4* __restrict__ rec, uint32_t item) {
    const float z = rec[4 * (size_t)item + 3].y;
    return ((uint64_t)__float_as_uint(z) << 32) | item;
}

// stable radix sort of keys[0, n) by one CTA (a multiple of 32 threads);
// result in keys
__device__ __noinline__ void block_radix_sort_global(uint64_t* keys, uint64_t* tmp, int n) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t offs[256];
    __shared__ int skip;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x, nw = nt >> 5;
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = pass * 8;
        for (int d = tid; d < 256; d += nt) hist[d] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += nt) atomicAdd(&hist[(src[i] >> shift) & 255u], 1u);
        __syncthreads();
        if (tid == 0) {
            uint32_t run = 0;
            skip = 0;
            for (int d = 0; d < 256; ++d) {
                if (hist[d] == (uint32_t)n) skip = 1;
                offs[d] = run;
                run += hist[d];
            }
        }
        __syncthreads();
        if (skip) continue;  // every key has the same digit: order unchanged
        for (int base = 0; base < n; base += nt) {
            const int i = base + tid;
            const bool ok = i < n;
            const uint64_t k = ok ? src[i] : 0ull;
            const uint32_t d = ok ? (uint32_t)((k >> shift) & 255u) : 256u + (uint32_t)lane;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int leader = __ffs(peers) - 1;
            for (int w = 0; w < nw; ++w) {  // warps in order keep the sort stable
                if (wid == w && ok) {
                    dst[offs[d] + rank] = k;
                }
                __syncwarp();
                if (wid == w && ok && lane == leader) offs[d] += __popc(peers);
                __syncthreads();
            }
        }
        __syncthreads();
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != keys)
        for (int i = tid; i < n; i += nt) keys[i] = src[i];
    __syncthreads();
}

}  // namespace

// Sorts tile t's list in place and writes its warp masks.  Called by every
// thread of the CTA (any multiple of 32 threads); sk, smask and spos are
// SORT_CAP entries of shared memory.  Returns with the list and masks in
// global memory written by this CTA (the caller synchronises before reading
// them back).
static __device__ __noinline__ void sort_tile(const Cams& cams, const RParams& P, const float4* __restrict__ rec,
                                          const BinRec* __restrict__ binrec, const int2* __restrict__ ranges,
                                          uint32_t* list, const uint32_t* __restrict__ unb_list,
                                          uint64_t* __restrict__ scratch, uint32_t* masks, Status* stw, int t,
                                          uint64_t* sk, uint32_t* smask, uint16_t* spos) {
    const int2 rg = checked_range(ranges, t, P.pair_cap, stw);
    const int n = rg.y - rg.x;
    if (n <= 0) return;
    const int view = view_of_tile(cams, t);
    const CamDev& cam = cams.c[view];
    const int lt = t - cam.tile_off;
    const int tx0 = (lt % cam.tiles_x) * P.ts, ty0 = (lt / cam.tiles_x) * P.ts;
    const int nu = (int)stw->unb_cnt[view];
    if (!in_bounds(stw, SITE_VIS_LIST, nu, ((int64_t)n < P.N ? (int64_t)n : P.N) + 1)) return;
    const int nb = n - nu;
    const uint32_t* ul = unb_list + (int64_t)view * P.N;
    const int tid = threadIdx.x, nt = blockDim.x;
    // the i-th item of the tile (bounded items, then the view's unbounded ones), checked
    auto item_at = [&](int i) -> uint32_t {
        const uint32_t it = i < nb ? list[rg.x + i] : ul[i - nb];
        return in_bounds(stw, SITE_ITEM, it, P.n_items) ? it : 0u;
    };
    if (n <= SORT_CAP) {
        // Lists in shared memory, in 32-key chunks (padding keys ~0 are larger
        // than every key: depth bits < 0x7f800000):
        //  A. each pair's key and warp mask (the mask does not depend on the
        //     order, so it is formed here, beside the key's gather);
        //  B. each warp sorts its chunks in registers (bitonic network over
        //     the lanes), carrying each key's position in the list;
        //  C. a key's rank is its place in its chunk plus, per other chunk,
        //     the number of smaller keys there (a 32-way binary search); the
        //     keys are unique, so the ranks are a permutation.
        const int nch = (n + 31) >> 5, lane = tid & 31, w = tid >> 5;
#pragma unroll 2
        for (int i = tid; i < (nch << 5); i += nt) {
            uint64_t k = ~0ull;
            if (i < n) {
                const uint32_t item = item_at(i);
                k = sort_key(rec, item);
                smask[i] = P.lowpass ? warp_block_mask<true>(binrec + item, P.ts, tx0, ty0)
                                     : warp_block_mask<false>(binrec + item, P.ts, tx0, ty0);
            }
            sk[i] = k;
        }
        __syncthreads();
        for (int c = w; c < nch; c += nt >> 5) {
            uint64_t k = sk[(c << 5) + lane];
            int pos = (c << 5) + lane;
#pragma unroll
            for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    const uint64_t ok = __shfl_xor_sync(0xffffffffu, k, j);
                    const int op = __shfl_xor_sync(0xffffffffu, pos, j);
                    const bool keep_min = ((lane & kk) == 0) == ((lane & j) == 0);  // ascending runs
                    const bool take = keep_min ? ok < k : ok > k;
                    k = take ? ok : k;
                    pos = take ? op : pos;
                }
            }
            sk[(c << 5) + lane] = k;
            spos[(c << 5) + lane] = (uint16_t)pos;
        }
        __syncthreads();
        for (int q = tid; q < n; q += nt) {
            const uint64_t k = sk[q];
            const int c = q >> 5;
            int rank = q & 31;
            for (int c2 = 0; c2 < nch; ++c2) {
                if (c2 == c) continue;
                const uint64_t* a = sk + (c2 << 5);
                int cnt = a[31] < k ? 32 : 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) cnt += (cnt < 32 && a[cnt + step - 1] < k) ? step : 0;
                rank += cnt;
            }
            list[rg.x + rank] = (uint32_t)k;
            masks[rg.x + rank] = smask[spos[q]];
        }
        return;
    }
    uint64_t* keys = scratch + rg.x;
    uint64_t* tmp = scratch + P.pair_cap + rg.x;
    for (int i = tid; i < n; i += nt) keys[i] = sort_key(rec, item_at(i));
    __syncthreads();
    block_radix_sort_global(keys, tmp, n);
    for (int i = tid; i < n; i += nt) {
        const uint32_t item = (uint32_t)keys[i];
        list[rg.x + i] = item;
        masks[rg.x + i] = (P.lowpass ? warp_block_mask<true>(binrec + item, P.ts, tx0, ty0)
                                     : warp_block_mask<false>(binrec + item, P.ts, tx0, ty0));
    }
}

}  // namespace fss
