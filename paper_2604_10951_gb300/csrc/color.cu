// Per-item view-dependent colours (Sec. 3.1) for the spherical-harmonic
// colour mode, one thread per visible (view, surfel) item:
//   k_sh_dir   (binning, which has the centres): the unit direction d from
//              the view's camera centre to the surfel centre -> REG_DIR;
//   k_sh_color (forward, which has the coefficients): c = max(0, sum_b k_b
//              Y_b(d) + 1/2) -> REG_COLOR [items, 3], which the render
//              kernels read in place of the per-surfel RGB input.
// The items are those binning listed as visible (bounded narrow and wide
// ones, and the unbounded ones of each view); no other item's colour is ever
// read.
#include "color.cuh"
#include "kernels.cuh"

namespace fss {

// i-th visible item: narrow, wide, then each view's unbounded ones
__device__ __forceinline__ uint32_t visible_item(int64_t i, uint32_t nvis, uint32_t nwide, const uint32_t* vis_list,
                                                 const uint32_t* wide_list, const uint32_t* unb_list, const Status* st,
                                                 int64_t N) {
    Status* const stw = const_cast<Status*>(st);  // check build: failed index checks are recorded here
    if (!in_bounds(stw, SITE_VIS_LIST, i, N * FSS_MAX_CAMS)) return ~0u;
    if (i < nvis) return vis_list[i];
    if (i < (int64_t)nvis + nwide) return wide_list[i - nvis];
    uint32_t k = (uint32_t)(i - nvis - nwide);
    int v = 0;
    while (v < FSS_MAX_CAMS && k >= st->unb_cnt[v]) k -= st->unb_cnt[v++];
    if (!in_bounds(stw, SITE_VIS_LIST, v, FSS_MAX_CAMS) || !in_bounds(stw, SITE_VIS_LIST, k, N)) return ~0u;
    return unb_list[(int64_t)v * N + k];
}

__global__ void __launch_bounds__(256) k_sh_dir(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                const uint32_t* __restrict__ vis_list,
                                                const uint32_t* __restrict__ wide_list,
                                                const uint32_t* __restrict__ unb_list, const float* __restrict__ means,
                                                float4* __restrict__ dir, const Status* __restrict__ st) {
    if (st->err) return;
    const uint32_t nvis = st->nvis, nwide = st->nwide;
    uint32_t nunb = 0;
    for (int v = 0; v < cams.n; ++v) nunb += st->unb_cnt[v];
    const int64_t n = (int64_t)nvis + nwide + nunb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t item = visible_item(i, nvis, nwide, vis_list, wide_list, unb_list, st, P.N);
        if (!in_bounds(const_cast<Status*>(st), SITE_ITEM, item, P.n_items)) continue;
        const int view = (int)((int64_t)item / P.N);
        const int64_t s = (int64_t)item - (int64_t)view * P.N;
        float ox, oy, oz;
        cam_centre(cams.c[view], ox, oy, oz);
        const float vx = means[3 * s] - ox, vy = means[3 * s + 1] - oy, vz = means[3 * s + 2] - oz;
        const float ir = rsqrtf(vx * vx + vy * vy + vz * vz);
        dir[item] = make_float4(vx * ir, vy * ir, vz * ir, ir);
    }
}

__global__ void __launch_bounds__(256) k_sh_color(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                  const uint32_t* __restrict__ vis_list,
                                                  const uint32_t* __restrict__ wide_list,
                                                  const uint32_t* __restrict__ unb_list,
                                                  const float4* __restrict__ dir, const float* __restrict__ coef,
                                                  float* __restrict__ color, const Status* __restrict__ st) {
    if (st->err) return;
    const uint32_t nvis = st->nvis, nwide = st->nwide;
    uint32_t nunb = 0;
    for (int v = 0; v < cams.n; ++v) nunb += st->unb_cnt[v];
    const int64_t n = (int64_t)nvis + nwide + nunb;
    const int nb = (P.sh_deg + 1) * (P.sh_deg + 1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t item = visible_item(i, nvis, nwide, vis_list, wide_list, unb_list, st, P.N);
        if (!in_bounds(const_cast<Status*>(st), SITE_ITEM, item, P.n_items)) continue;
        const int64_t s = (int64_t)item - (int64_t)((int64_t)item / P.N) * P.N;
        const float4 d = dir[item];
        float Y[16];
        sh_basis(P.sh_deg, d.x, d.y, d.z, Y);
        const float* k = coef + s * nb * 3;
        float c[3] = {0.5f, 0.5f, 0.5f};
        for (int b = 0; b < nb; ++b) {
            c[0] = fmaf(k[3 * b], Y[b], c[0]);
            c[1] = fmaf(k[3 * b + 1], Y[b], c[1]);
            c[2] = fmaf(k[3 * b + 2], Y[b], c[2]);
        }
        color[3 * (int64_t)item] = fmaxf(c[0], 0.0f);
        color[3 * (int64_t)item + 1] = fmaxf(c[1], 0.0f);
        color[3 * (int64_t)item + 2] = fmaxf(c[2], 0.0f);
    }
}

cudaError_t launch_sh_dir(const Cams& cams, const RParams& P, const uint32_t* vis_list, const uint32_t* wide_list,
                          const uint32_t* unb_list, const float* means, float4* dir, const Status* st, int num_sms,
                          cudaStream_t stream) {
    k_sh_dir<<<num_sms * 4, 256, 0, stream>>>(cams, P, vis_list, wide_list, unb_list, means, dir, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) kernel_mark(stream);
    return e;
}

cudaError_t launch_sh_color(const Cams& cams, const RParams& P, const uint32_t* vis_list, const uint32_t* wide_list,
                            const uint32_t* unb_list, const float4* dir, const float* coef, float* color,
                            const Status* st, int num_sms, cudaStream_t stream) {
    k_sh_color<<<num_sms * 4, 256, 0, stream>>>(cams, P, vis_list, wide_list, unb_list, dir, coef, color, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) kernel_mark(stream);
    return e;
}

}  // namespace fss
