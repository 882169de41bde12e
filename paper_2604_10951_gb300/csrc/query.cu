// Query-guided instance labels (Sec. 3.3) on the 5th-generation tensor cores.
//
// For every scene Gaussian g and instance query q:
//   S = sigmoid(f_q . f_ins(g)),  D = exp(-1/2 d^T Sigma_q^-1 d), d = p_g - p_q,
//   A = S D,  l_ins(g) = softmax over q of A.
// The similarity logits f_ins F_q^T are a dense [N, dim] x [dim, nq]
// contraction, so they run as tcgen05 MMAs: one CTA of 4 warps takes 128
// Gaussians at a time (MMA M = 128, N = nq, K = dim in steps of 16, BF16
// operands, FP32 accumulator in tensor memory).  The epilogue reads the
// accumulator back with tcgen05.ld, one TMEM lane (= one Gaussian) per
// thread, so the softmax over the queries needs no cross-thread reduction:
// pass 1 turns each logit into exp(A) and writes it back to tensor memory
// while summing, pass 2 reads exp(A) again and stores exp(A) / sum.
//
// Shared-memory operands use the no-swizzle K-major layout of 8 x 16-byte
// core matrices: element (r, k) of a [rows, dim] operand sits at byte
// ((r / 8) * (dim / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, i.e. a
// leading-dimension (K) step of 128 bytes between core matrices and a
// stride-dimension (row-group) step of dim * 16 bytes.
//
// Every wait on the MMA's mbarrier is bounded: on expiry the kernel raises
// the caller's error word, stops taking tiles, frees its tensor memory and
// returns.
#include "fss_internal.cuh"
#include "kernels.cuh"
#include "render_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace fss {

namespace {

constexpr int QM = 128;        // Gaussians per tile (MMA M)
constexpr int QTHREADS = 128;  // warp w reads TMEM lanes 32 w .. 32 w + 31
constexpr int QWAIT = 1 << 22; // try_wait rounds before giving up
constexpr float QLOG2E = 1.4426950408889634f;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (row-group)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(QM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < QWAIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

// Operand staging in the core-matrix layout.  Chunk j of a tile (16 bytes,
// 8 BF16) goes to row r = 8 (j / (8 KC)) + j % 8 and K-chunk c = (j / 8) % KC:
// the 8 threads of a shared-memory store phase write the 8 rows of one core
// matrix (128 consecutive bytes, no bank conflict), and a warp still reads
// 8 whole consecutive rows of global memory.
template <int KC>
__device__ __forceinline__ int stage_row(int j) { return ((j / (8 * KC)) << 3) | (j & 7); }
template <int KC>
__device__ __forceinline__ int stage_col(int j) { return (j >> 3) % KC; }
template <int KC>
__device__ __forceinline__ uint32_t stage_off(int j) {
    const int r = stage_row<KC>(j), c = stage_col<KC>(j);
    return ((uint32_t)((r >> 3) * KC + c) << 7) + ((uint32_t)(r & 7) << 4);
}

// rows [r0, r0 + nrows) of a row-major [*, 8 KC] BF16 matrix (rows past
// `valid` are zero) into the core-matrix layout at dst
template <int KC>
__device__ __forceinline__ void stage_rows(unsigned char* dst, const __nv_bfloat16* __restrict__ src, int64_t r0,
                                           int nrows, int64_t valid) {
    for (int j = threadIdx.x; j < nrows * KC; j += blockDim.x) {
        const int r = stage_row<KC>(j), c = stage_col<KC>(j);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r0 + r < valid) v = __ldg(reinterpret_cast<const uint4*>(src + (r0 + r) * (8 * KC)) + c);
        *reinterpret_cast<uint4*>(dst + stage_off<KC>(j)) = v;
    }
}

// this thread's KC chunks of a 128-row tile (chunk j = tid + i * 128), into registers
template <int KC>
__device__ __forceinline__ void load_tile(uint4 (&v)[KC], const __nv_bfloat16* __restrict__ src, int64_t r0,
                                          int64_t valid) {
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        const int j = threadIdx.x + i * QTHREADS;
        const int r = stage_row<KC>(j), c = stage_col<KC>(j);
        v[i] = make_uint4(0u, 0u, 0u, 0u);
        if (r0 + r < valid) v[i] = __ldg(reinterpret_cast<const uint4*>(src + (r0 + r) * (8 * KC)) + c);
    }
}

template <int KC>
__global__ void __launch_bounds__(QTHREADS, KC <= 4 ? 8 : 1) k_query_labels(int64_t N, int nq, int ncols,
                                                           const __nv_bfloat16* __restrict__ f_ins,
                                                           const float* __restrict__ means,
                                                           const __nv_bfloat16* __restrict__ f_q,
                                                           const float* __restrict__ p_q,
                                                           const float* __restrict__ prec, void* __restrict__ out,
                                                           int out_bf16, int32_t* __restrict__ err) {
    constexpr int dim = 8 * KC;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                                  // [128 x dim] core matrices
    unsigned char* sB = sA + (size_t)QM * dim * 2;             // [nq x dim] core matrices
    // [nq][3] float4: (p_q, -log2(e)/2 xx), (-log2(e)/2 yy, zz; -log2(e) xy, xz), (-log2(e) yz, 0, 0, 0),
    // so that D = 2^(quadratic form in d)
    float4* s_qp = reinterpret_cast<float4*>(sB + (size_t)nq * dim * 2);
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (N + QM - 1) / QM;

    // queries: operand B and the per-query proximity parameters, once per CTA
    stage_rows<KC>(sB, f_q, 0, nq, nq);
    for (int q = tid; q < nq; q += blockDim.x) {
        const float h = -0.5f * QLOG2E, f = -QLOG2E;
        const float* P = prec + 6 * q;
        s_qp[3 * q] = make_float4(p_q[3 * q], p_q[3 * q + 1], p_q[3 * q + 2], h * P[0]);
        s_qp[3 * q + 1] = make_float4(h * P[1], h * P[2], f * P[3], f * P[4]);
        s_qp[3 * q + 2] = make_float4(f * P[5], 0.0f, 0.0f, 0.0f);
    }
    if (tid == 0) {
        s_abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // visible to the MMA's arrive
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes, column 0
    const uint32_t bar = smem_u32(&s_bar);
    const uint32_t idesc = mma_idesc(nq);
    uint32_t phase = 0;

    // the next tile's operand rows and Gaussian centre, loaded while the
    // current tile is in the tensor core and the epilogue
    uint4 pre[KC];
    float npx = 0.0f, npy = 0.0f, npz = 0.0f;
    int64_t tile = blockIdx.x;
    if (tile < ntiles) {
        load_tile<KC>(pre, f_ins, tile * QM, N);
        const int64_t g = tile * QM + tid;
        if (g < N) { npx = means[3 * g]; npy = means[3 * g + 1]; npz = means[3 * g + 2]; }
    }
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t g0 = tile * QM;
#pragma unroll
        for (int i = 0; i < KC; ++i) *reinterpret_cast<uint4*>(sA + stage_off<KC>(tid + i * QTHREADS)) = pre[i];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor core reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < KC / 2; ++s) {  // K = 16 per MMA: two 16-byte chunks
                const uint64_t da = smem_desc(smem_u32(sA) + 256u * s, 128u, KC * 128u);
                const uint64_t db = smem_desc(smem_u32(sB) + 256u * s, 128u, KC * 128u);
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(s)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        // this tile's centre (the thread's TMEM lane is tid), then the next tile's loads
        const float px = npx, py = npy, pz = npz;
        const int64_t nt = tile + gridDim.x;
        if (nt < ntiles) {
            load_tile<KC>(pre, f_ins, nt * QM, N);
            const int64_t gn = nt * QM + tid;
            if (gn < N) { npx = means[3 * gn]; npy = means[3 * gn + 1]; npz = means[3 * gn + 2]; }
        }
        if (!mbar_wait(bar, phase)) s_abort = 1;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (s_abort) break;

        // epilogue: this thread's Gaussian is TMEM lane 32 warp + lane = tid
        const int64_t g = g0 + tid;
        const bool live = g < N;
        float sum = 0.0f;
        for (int c0 = 0; c0 < nq; c0 += 16) {
            float v[16];
            tmem_ld16(tlane + c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float4 a = s_qp[3 * (c0 + i)], b = s_qp[3 * (c0 + i) + 1], c = s_qp[3 * (c0 + i) + 2];
                const float S = rcp_approx(1.0f + ex2_approx(-QLOG2E * v[i]));  // sigmoid
                const float dx = px - a.x, dy = py - a.y, dz = pz - a.z;
                // log2 D = -log2(e)/2 d^T Sigma^-1 d
                const float l2d = fmaf(fmaf(a.w, dx, fmaf(b.z, dy, b.w * dz)), dx,
                                       fmaf(fmaf(b.x, dy, c.x * dz), dy, b.y * dz * dz));
                const float e = ex2_approx(QLOG2E * S * ex2_approx(l2d));  // exp(A), A = S D
                v[i] = e;
                sum += e;
            }
            tmem_st16(tlane + c0, v);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        const float inv = 1.0f / sum;
        for (int c0 = 0; c0 < nq; c0 += 16) {
            float v[16];
            tmem_ld16(tlane + c0, v);
            if (!live) continue;
            if (out_bf16) {
                uint4 w[2];
                uint32_t* h = reinterpret_cast<uint32_t*>(w);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * i] * inv, v[2 * i + 1] * inv);
                    h[i] = *reinterpret_cast<const uint32_t*>(&b2);
                }
                uint4* o = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + g * nq + c0);
                o[0] = w[0];
                o[1] = w[1];
            } else {
                float4* o = reinterpret_cast<float4*>(static_cast<float*>(out) + g * nq + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    o[i] = make_float4(v[4 * i] * inv, v[4 * i + 1] * inv, v[4 * i + 2] * inv, v[4 * i + 3] * inv);
            }
        }
        // every lane's reads of the accumulator and of sA are done before the
        // next tile's stores and MMA
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (s_abort && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

template <int KC>
cudaError_t launch_kc(int64_t N, int nq, const void* f_ins, const float* means, const void* f_q, const float* p_q,
                      const float* prec, void* out, int out_bf16, int32_t* err, int num_sms, cudaStream_t stream) {
    int ncols = 32;
    while (ncols < nq) ncols <<= 1;
    const size_t smem = query_labels_smem(nq, 8 * KC);
    auto kern = k_query_labels<KC>;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // resident CTAs per SM from the kernel's registers and shared memory (the
    // occupancy query answers 1 for this tensor-memory kernel), at most the
    // number whose tensor-memory columns fit the SM's 512 together
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, smem_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    const int regs = ((std::max(fa.numRegs, 1) + 7) & ~7) * QTHREADS;
    int per_sm = std::min({2048 / QTHREADS, 65536 / regs, smem_sm / (int)(smem + fa.sharedSizeBytes + 1024),
                           512 / ncols});
    per_sm = std::max(1, per_sm);
    const int64_t ntiles = (N + QM - 1) / QM;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * num_sms);
    kern<<<grid, QTHREADS, smem, stream>>>(N, nq, ncols, static_cast<const __nv_bfloat16*>(f_ins), means,
                                           static_cast<const __nv_bfloat16*>(f_q), p_q, prec, out, out_bf16, err);
    e = cudaGetLastError();
    if (e == cudaSuccess) kernel_mark(stream);
    return e;
}

}  // namespace

size_t query_labels_smem(int nq, int dim) { return (size_t)QM * dim * 2 + (size_t)nq * dim * 2 + (size_t)nq * 48; }

cudaError_t launch_query_labels(int64_t N, int nq, int dim, const void* f_ins, const float* means, const void* f_q,
                                const float* p_q, const float* prec, void* out, int out_bf16, int32_t* err,
                                int num_sms, cudaStream_t stream) {
    if (N <= 0) return cudaSuccess;
    switch (dim) {
        case 16: return launch_kc<2>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
        case 32: return launch_kc<4>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
        case 48: return launch_kc<6>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
        case 64: return launch_kc<8>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
        case 80: return launch_kc<10>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
        case 96: return launch_kc<12>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
        case 112: return launch_kc<14>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
        default: return launch_kc<16>(N, nq, f_ins, means, f_q, p_q, prec, out, out_bf16, err, num_sms, stream);
    }
}

}  // namespace fss
