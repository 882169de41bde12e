// Depth-sort kernel: one CTA of SORT_THREADS threads per tile runs
// sort_tile (sort.cuh) on its tile.
#include "sort.cuh"

namespace fss {

__global__ void __launch_bounds__(SORT_THREADS, 8) k_tile_sort(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                   const float4* __restrict__ rec, const BinRec* __restrict__ binrec,
                                                   const int2* __restrict__ ranges, uint32_t* __restrict__ list,
                                                   const uint32_t* __restrict__ unb_list,
                                                   uint64_t* __restrict__ scratch, uint32_t* __restrict__ masks,
                                                   const Status* __restrict__ st) {
    __shared__ __align__(16) uint64_t sk[SORT_CAP];
    __shared__ uint32_t smask[SORT_CAP];
    __shared__ uint16_t spos[SORT_CAP];
    if (st->err) return;
    Status* const stw = const_cast<Status*>(st);  // check build: failed index checks are recorded here
    // index order: measured faster here than the heavy-first order
    sort_tile(cams, P, rec, binrec, ranges, list, unb_list, scratch, masks, stw, blockIdx.x, sk, smask, spos);
}

}  // namespace fss
