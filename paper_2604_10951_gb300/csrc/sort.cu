// Depth sort of each tile's surfel list (the paper composites the surfels
// in depth order, Sec. 3.1).
//
// Binning leaves every tile's range of the pair list filled in arbitrary
// order (bounded items first, then the view's unbounded items are appended
// here).  One CTA per tile sorts its range by the 64-bit key
//   (binary32 bits of the item's camera depth) << 32 | item index,
// which is unique, so the order is total and deterministic.  Depths are
// positive, so their bit patterns order like the numbers.
//   - up to blockDim.x keys: rank sort (each thread counts the smaller keys);
//   - up to SORT_CAP keys: bitonic sort in shared memory;
//   - longer lists: stable LSD radix sort (8-bit digits) by the same CTA
//     in a global scratch range of the same offsets.
// With the sorted item, each pair gets the mask of the tile's warps (8 x 4
// pixel blocks) that its footprint reaches, which the render passes use
// to skip a surfel warp by warp.
#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"

namespace fss {

namespace {

__device__ __forceinline__ uint64_t make_key(const float4* __restrict__ rec, uint32_t item) {
    const float z = rec[4 * (size_t)item + 3].y;
    return ((uint64_t)__float_as_uint(z) << 32) | item;
}

// stable radix sort of keys[0, n) by one CTA of 256 threads; result in keys
__device__ void block_radix_sort_global(uint64_t* keys, uint64_t* tmp, int n) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t offs[256];
    __shared__ int skip;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = pass * 8;
        hist[tid] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += 256) atomicAdd(&hist[(src[i] >> shift) & 255u], 1u);
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
        for (int base = 0; base < n; base += 256) {
            const int i = base + tid;
            const bool ok = i < n;
            const uint64_t k = ok ? src[i] : 0ull;
            const uint32_t d = ok ? (uint32_t)((k >> shift) & 255u) : 256u + (uint32_t)lane;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int leader = __ffs(peers) - 1;
            for (int w = 0; w < 8; ++w) {  // warps in order keep the sort stable
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
        for (int i = tid; i < n; i += 256) keys[i] = src[i];
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(256) k_tile_sort(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                   const float4* __restrict__ rec, const BinRec* __restrict__ binrec,
                                                   const int2* __restrict__ ranges, uint32_t* __restrict__ list,
                                                   const uint32_t* __restrict__ unb_list,
                                                   uint64_t* __restrict__ scratch, uint32_t* __restrict__ masks,
                                                   const Status* __restrict__ st) {
    __shared__ uint64_t sk[SORT_CAP];
    if (st->err) return;
    Status* const stw = const_cast<Status*>(st);  // check build: failed index checks are recorded here
    const int t = blockIdx.x;  // index order: measured faster here than the heavy-first order
    const int2 rg = checked_range(ranges, t, P.pair_cap, stw);
    const int n = rg.y - rg.x;
    if (n <= 0) return;
    const int view = view_of_tile(cams, t);
    const CamDev& cam = cams.c[view];
    const int lt = t - cam.tile_off;
    const int tx0 = (lt % cam.tiles_x) * P.ts, ty0 = (lt / cam.tiles_x) * P.ts;
    const int nu = (int)st->unb_cnt[view];
    if (!in_bounds(stw, SITE_VIS_LIST, nu, ((int64_t)n < P.N ? (int64_t)n : P.N) + 1)) return;
    const int nb = n - nu;
    const uint32_t* ul = unb_list + (int64_t)view * P.N;
    const int tid = threadIdx.x;
    // the i-th item of the tile (bounded items, then the view's unbounded ones), checked
    auto item_at = [&](int i) -> uint32_t {
        const uint32_t it = i < nb ? list[rg.x + i] : ul[i - nb];
        return in_bounds(stw, SITE_ITEM, it, P.n_items) ? it : 0u;
    };
    if (n <= (int)blockDim.x) {
        // short list: rank of each key = number of smaller keys (keys are
        // unique, so the ranks are a permutation); one barrier instead of a
        // network of them
        uint64_t key = ~0ull;
        if (tid < n) key = make_key(rec, item_at(tid));
        sk[tid] = key;
        __syncthreads();
        if (tid < n) {
            int rank = 0;
            for (int j = 0; j < n; ++j) rank += sk[j] < key ? 1 : 0;
            const uint32_t item = (uint32_t)key;
            list[rg.x + rank] = item;
            masks[rg.x + rank] = (P.lowpass ? warp_block_mask<true>(binrec + item, P.ts, tx0, ty0)
                                           : warp_block_mask<false>(binrec + item, P.ts, tx0, ty0));
        }
        return;
    }
    if (n <= SORT_CAP) {
        int m = 1;
        while (m < n) m <<= 1;
        for (int i = tid; i < m; i += blockDim.x) {
            uint64_t k = ~0ull;
            if (i < n) k = make_key(rec, item_at(i));
            sk[i] = k;
        }
        __syncthreads();
        for (int k = 2; k <= m; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < (m >> 1); i += blockDim.x) {
                    const int l = ((i & ~(j - 1)) << 1) | (i & (j - 1));  // j is a power of two
                    const int r = l + j;
                    const bool up = (l & k) == 0;
                    const uint64_t a = sk[l], b = sk[r];
                    if ((a > b) == up) { sk[l] = b; sk[r] = a; }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i < n; i += blockDim.x) {
            const uint32_t item = (uint32_t)sk[i];
            list[rg.x + i] = item;
            masks[rg.x + i] = (P.lowpass ? warp_block_mask<true>(binrec + item, P.ts, tx0, ty0)
                                           : warp_block_mask<false>(binrec + item, P.ts, tx0, ty0));
        }
        return;
    }
    uint64_t* keys = scratch + rg.x;
    uint64_t* tmp = scratch + P.pair_cap + rg.x;
    for (int i = tid; i < n; i += blockDim.x) keys[i] = make_key(rec, item_at(i));
    __syncthreads();
    block_radix_sort_global(keys, tmp, n);
    for (int i = tid; i < n; i += blockDim.x) {
        const uint32_t item = (uint32_t)keys[i];
        list[rg.x + i] = item;
        masks[rg.x + i] = (P.lowpass ? warp_block_mask<true>(binrec + item, P.ts, tx0, ty0)
                                           : warp_block_mask<false>(binrec + item, P.ts, tx0, ty0));
    }
}

}  // namespace fss
