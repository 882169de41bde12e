// Training loss used by the forward+backward workload and its gradient, in
// one pass:  L = w_f * mean((F - F_t)^2) + w_c * mean(|rgb - rgb_t|)
// (an L2 feature term standing in for the semantic/instance losses and the
// L1 part of the photometric loss, Sec. 3.5).  Writes dL/dF (in F's dtype)
// and dL/drgb, and adds L into a device double.
#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"

namespace fss {

template <typename OT>
__global__ void __launch_bounds__(256) k_loss(int64_t n_pix, int C, const OT* __restrict__ F,
                                              const float* __restrict__ rgb, const OT* __restrict__ Ft,
                                              const float* __restrict__ rgbt, float wf, float wc,
                                              OT* __restrict__ dF, float* __restrict__ drgb, double* __restrict__ loss) {
    constexpr int E = FeatVec<OT>::E;
    const int nvec = C / E;
    const int64_t nf = n_pix * nvec, nc = n_pix * 3;
    const float sf = 2.0f * wf / (float)(n_pix * C), sc = wc / (float)nc;
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // U grid-stride steps at a time, their loads all issued first (enough
    // bytes in flight for the copy rate); the sum keeps the steps' order
    constexpr int U = 4;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nf; i0 += U * stride) {
        typename FeatVec<OT>::Raw ra[U], rb[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < nf) {  // read once: streaming loads, so that L2 keeps what the backward reads next
                ra[u] = FeatVec<OT>::raw_cs(F + i * E);
                rb[u] = FeatVec<OT>::raw_cs(Ft + i * E);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= nf) break;
            float2 a2[E / 2], b2[E / 2];
            FeatVec<OT>::unpack2(ra[u], a2);
            FeatVec<OT>::unpack2(rb[u], b2);
            float g[E];
#pragma unroll
            for (int e = 0; e < E / 2; ++e) {
                const float d0 = a2[e].x - b2[e].x, d1 = a2[e].y - b2[e].y;
                acc = fmaf(d0, d0, acc);
                acc = fmaf(d1, d1, acc);
                g[2 * e] = sf * d0;
                g[2 * e + 1] = sf * d1;
            }
            store_vec<E>(dF, i * E, g, sizeof(OT) == 4 ? FSS_F32 : FSS_BF16);
        }
    }
    float accf = acc * wf / (float)(n_pix * C), accc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += stride) {
        const float d = __ldcs(rgb + i) - __ldcs(rgbt + i);
        accc += fabsf(d);
        drgb[i] = d > 0.0f ? sc : (d < 0.0f ? -sc : 0.0f);
    }
    float v = accf + accc * wc / (float)nc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ float s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s[k];
        atomicAdd(loss, t);
    }
}

cudaError_t launch_loss(int64_t n_pix, int C, int dtype, const void* F, const float* rgb, const void* Ft,
                        const float* rgbt, float wf, float wc, void* dF, float* drgb, double* loss, int num_sms,
                        cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (dtype == FSS_BF16)
        k_loss<__nv_bfloat16><<<num_sms * 4, 256, 0, s>>>(n_pix, C, (const __nv_bfloat16*)F, rgb,
                                                          (const __nv_bfloat16*)Ft, rgbt, wf, wc, (__nv_bfloat16*)dF,
                                                          drgb, loss);
    else
        k_loss<float><<<num_sms * 4, 256, 0, s>>>(n_pix, C, (const float*)F, rgb, (const float*)Ft, rgbt, wf, wc,
                                                  (float*)dF, drgb, loss);
    e = cudaGetLastError();
    if (e == cudaSuccess) kernel_mark(s);
    return e;
}

}  // namespace fss
