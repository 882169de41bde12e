// Device helpers shared by the forward and backward render kernels.  The
// per-evaluation arithmetic lives here once, so the backward replay takes
// exactly the forward's skip decisions.
#pragma once

#include "fss_internal.cuh"
#include "kernels.cuh"

#include <climits>

namespace fss {

constexpr int BATCH = 256;   // staged records per batch (Top-K kernels)
constexpr int FBATCH = 64;   // staged records + feature rows per batch (full kernels)
constexpr float NEG_HALF_LOG2E = -0.72134752044448170f;  // exp(-r/2) = 2^(r * this)

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Ray-splat intersection and opacity of one staged surfel at pixel point
// (pxf, pyf) (Eq. 2 density, alpha before the clamp).  Returns false when
// the surfel is skipped (alpha below alpha_min, hit at or behind the near
// plane, or a non-finite intersection).
struct Hit {
    float X, Y, u, v, inv, G, alpha_raw;  // G = exp(-(u^2+v^2)/2), alpha_raw = o G
    bool scr;                             // low-pass: the screen-space term gave G
};

// LP instances also apply the 2DGS low-pass filter when `lowpass` is set:
// rho = min(u^2 + v^2, 2 (X^2 + Y^2)), (X, Y) the pixel point about the
// projected centre; the screen term takes the centre's depth, which passed
// the near plane at binning, so it skips the near-plane test.
template <bool LP = false>
__device__ __forceinline__ bool eval_splat(const float4& A, const float4& B, const float4& Cq, float o, float pxf,
                                           float pyf, float alpha_min, float near_plane, Hit& h, bool lowpass = false) {
    h.X = pxf - A.w;
    h.Y = pyf - B.w;
    const float c0 = fmaf(A.x, h.X, fmaf(A.y, h.Y, A.z));
    const float c1 = fmaf(B.x, h.X, fmaf(B.y, h.Y, B.z));
    const float c2 = fmaf(Cq.x, h.X, fmaf(Cq.y, h.Y, Cq.z));
    h.inv = rcp_approx(c2);
    h.u = c0 * h.inv;
    h.v = c1 * h.inv;
    float rho = fmaf(h.u, h.u, h.v * h.v);
    h.scr = false;
    if (LP && lowpass) {
        const float rs = 2.0f * fmaf(h.X, h.X, h.Y * h.Y);
        h.scr = !(rho <= rs);  // also for a non-finite object term
        rho = h.scr ? rs : rho;
    }
    h.G = ex2_approx(NEG_HALF_LOG2E * rho);
    h.alpha_raw = o * h.G;
    return (h.alpha_raw >= alpha_min) && ((LP && h.scr) || Cq.w * h.inv > near_plane);  // hit depth det / c2
}

// Camera-space unit normal of a surfel from its render record, turned to face
// the camera.  The third adjugate row m2 about the projected centre (xc, yc)
// is (S K)^-T (r_u r_v R_v n) up to a positive factor, with K the intrinsics
// and S the shift to the centre, so R_v n is along K^T S^T m2; it faces the
// camera when its dot product with the centre's ray (xc - cx)/fx,
// (yc - cy)/fy, 1 is not positive.
__device__ __forceinline__ float4 facing_normal(const float4& m2, float xc, float yc, const CamDev& cam) {
    const float nx = cam.fx * m2.x, ny = cam.fy * m2.y;
    const float nz = fmaf(cam.cx - xc, m2.x, fmaf(cam.cy - yc, m2.y, m2.z));
    const float dx = (xc - cam.cx) / cam.fx, dy = (yc - cam.cy) / cam.fy;
    const float inv = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    const float sg = fmaf(nx, dx, fmaf(ny, dy, nz)) > 0.0f ? -inv : inv;
    return make_float4(nx * sg, ny * sg, nz * sg, 0.0f);
}

template <typename FT>
struct FeatVec;

template <>
struct FeatVec<float> {
    static constexpr int E = 4;  // channels per 16-byte load
    using Raw = float4;          // one 16-byte chunk as loaded
    __device__ static __forceinline__ Raw raw(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
    // streaming load (evict-first: read once, leaves L2 to the data read next)
    __device__ static __forceinline__ Raw raw_cs(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
    __device__ static __forceinline__ void unpack2(const Raw& r, float2* o) {
        o[0] = make_float2(r.x, r.y);
        o[1] = make_float2(r.z, r.w);
    }
    __device__ static __forceinline__ void load(const float* p, float* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static __forceinline__ float one(const float* p) { return __ldg(p); }
    // E channels in pairs, as stored in this type (rounded like store_vec), and the 16-byte store
    __device__ static __forceinline__ Raw pack(const float2* v) { return make_float4(v[0].x, v[0].y, v[1].x, v[1].y); }
    __device__ static __forceinline__ void st(float* p, const Raw& r) { *reinterpret_cast<float4*>(p) = r; }
    // 16-byte shared-memory load
    __device__ static __forceinline__ void lds(const float* p, float* o) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};

template <>
struct FeatVec<__nv_bfloat16> {
    static constexpr int E = 8;
    using Raw = uint4;
    __device__ static __forceinline__ Raw raw(const __nv_bfloat16* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
    __device__ static __forceinline__ Raw raw_cs(const __nv_bfloat16* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
    __device__ static __forceinline__ void unpack2(const Raw& r, float2* o) {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = make_float2(__uint_as_float(w[k] << 16), __uint_as_float(w[k] & 0xffff0000u));
    }
    __device__ static __forceinline__ void load(const __nv_bfloat16* p, float* o) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[2 * k] = __uint_as_float(w[k] << 16);
            o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    __device__ static __forceinline__ Raw pack(const float2* v) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[k].x, v[k].y);
            w[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ static __forceinline__ void st(__nv_bfloat16* p, const Raw& r) { *reinterpret_cast<uint4*>(p) = r; }
    __device__ static __forceinline__ float one(const __nv_bfloat16* p) {
        return __uint_as_float(((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
    }
    __device__ static __forceinline__ void lds(const __nv_bfloat16* p, float* o) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[2 * k] = __uint_as_float(w[k] << 16);
            o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
};

// store E channels (E = 4 or 8) in the output dtype
template <int E>
__device__ __forceinline__ void store_vec(void* out, int64_t elem, const float* acc, int out_dtype) {
    if (out_dtype == FSS_F32) {
        float4* p = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + elem);
#pragma unroll
        for (int k = 0; k < E / 4; ++k) p[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
    } else {
        uint32_t w[E / 2];
#pragma unroll
        for (int k = 0; k < E / 2; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(acc[2 * k], acc[2 * k + 1]);
            w[k] = *reinterpret_cast<const uint32_t*>(&h);
        }
        __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(out) + elem;
        if (E == 8) *reinterpret_cast<uint4*>(b) = make_uint4(w[0], w[1], w[2], w[3]);
        else *reinterpret_cast<uint2*>(b) = make_uint2(w[0], w[1]);
    }
}

// 16-byte asynchronous global -> shared copy (bytes = 0: zero fill), its
// commit and the wait for all of this thread's copies
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Division by a divisor fixed for the whole kernel (d >= 1, 0 <= n < 2^24),
// without the ~20-instruction integer division: a float reciprocal guess
// corrected by one step either way.
struct FastDiv {
    int d;
    float r;
    __device__ __forceinline__ explicit FastDiv(int dd) : d(dd), r(1.0f / (float)dd) {}
    __device__ __forceinline__ int div(int n) const {
        int q = __float2int_rz(__int2float_rn(n) * r);
        q += ((q + 1) * d <= n) ? 1 : 0;
        q -= (q * d > n) ? 1 : 0;
        return q;
    }
};

// Pixel of thread `tid` in a TS x TS tile (TS in {8, 16, 32}): each warp
// owns an 8 x 4 pixel block, blocks row-major over the tile (TS / 8 per
// block row); lane l is pixel (l & 7, l >> 3) of its block.  Square-ish
// blocks let a warp skip surfels whose footprint misses its block in
// either direction.
template <int TS>
__device__ __forceinline__ int2 pixel_of(int tid) {
    constexpr int WX = TS / 8;
    const int w = tid >> 5, l = tid & 31;
    return make_int2(8 * (w % WX) + (l & 7), 4 * (w / WX) + (l >> 3));
}

// Mask of the warps of the ts x ts tile at (tile_x0, tile_y0) whose 8 x 4
// block (pixel_of) holds a pixel centre inside the surfel's binning ellipse
// (the opacity-aware cutoff with its slack, Sec. 3.2), or inside its pixel
// box when the footprint is unbounded.  Computed once per tile-surfel pair
// by the depth sort and read by the render passes.  Per 4-row strip the ellipse's x-extent is its
// left/right tangent point when that lies in the strip, else the root of
// A x^2 + 2(B y + D) x + (C y^2 + 2 E y + F) = 0 at the nearer strip edge;
// the extent is widened by a small margin, so the mask may keep a warp
// that misses but never drops one that is hit.  Skipping a warp therefore
// changes no result.  With the low-pass filter the extent also covers the
// screen disc of the binning record (radius^2 rd2 about the local origin),
// widened by 0.1 % in radius^2 and 0.05 pixel.
// The arithmetic is the approximate kind (reciprocal and square root to
// about 2^-22 relative; the extents move by far less than the margin) and
// has no branch inside a strip: the IEEE divide and square root each carry a
// slow-path branch, which kept the strips' chains from overlapping (about
// 900 cycles per strip where this takes a fraction).  The tangent points do
// not depend on the strip and are formed once.
template <bool LP>
__device__ __forceinline__ uint32_t warp_block_mask(const BinRec* __restrict__ rp, int ts, int tile_x0, int tile_y0) {
    const int WX = ts >> 3;
    const float4 q0 = __ldg(reinterpret_cast<const float4*>(rp));       // A B C D
    const float4 q1 = __ldg(reinterpret_cast<const float4*>(rp) + 1);   // E F X0 Y0
    const float4 q2 = __ldg(reinterpret_cast<const float4*>(rp) + 2);   // hx hy xc yc
    const int2 q3 = __ldg(reinterpret_cast<const int2*>(rp) + 6);       // pixel box (int16 x 4)
    const int px0 = (int)(int16_t)(q3.x & 0xffff), px1 = q3.x >> 16;
    const int py0 = (int)(int16_t)(q3.y & 0xffff), py1 = q3.y >> 16;
    const int flags = __ldg(&rp->flags);
    const bool unbounded = (flags & BR_UNBOUNDED) != 0;
    const bool ell = !LP || (flags & BR_ELL) != 0;
    const float rd2 = LP && (flags & BR_LOWPASS) ? __ldg(&rp->rd2) : -1.0f;  // low-pass screen disc
    const int x0 = max(px0, tile_x0), x1 = min(px1, tile_x0 + ts - 1);
    const int y0 = max(py0, tile_y0), y1 = min(py1, tile_y0 + ts - 1);
    if (x0 > x1 || y0 > y1) return 0u;
    const float A = q0.x, B = q0.y, Cc = q0.z, D = q0.w, E = q1.x, F = q1.y;
    const float X0 = q1.z, hx = q2.x, xc = q2.z, yc = q2.w;
    const float margin = 0.05f + 1e-3f * hx;
    const float iA = rcp_approx(A), iC = rcp_approx(Cc);
    const float Xs[2] = {X0 - hx, X0 + hx};
    const float Yt[2] = {-(B * Xs[0] + E) * iC, -(B * Xs[1] + E) * iC};
    // pixel indices held as floats (exact), so a strip needs no conversion
    const float fx0 = (float)x0, fx1 = (float)x1, fy0 = (float)y0, fy1 = (float)y1, ftx = (float)tile_x0;
    const int by0 = (y0 - tile_y0) >> 2, by1 = (y1 - tile_y0) >> 2;
    const float fs0 = (float)(tile_y0 + 4 * by0);  // first row of strip by0
    uint32_t m = 0u;
    // strips of 4 pixel rows, four at a time (each side's tangent and root
    // candidates are both formed and one is selected)
    for (int g = 0; g <= by1 - by0; g += 4) {
        const float fg = fs0 + (float)(4 * g);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int by = by0 + g + k;
            const float fr = fg + 4.0f * k;
            const float ra = fmaxf(fy0, fr), rb = fminf(fy1, fr + 3.0f);
            float ca = fx0, cb = fx1;
            bool keep = by <= by1;
            if (!unbounded) {
                const float Ya = (ra + 0.5f) - yc, Yb = (rb + 0.5f) - yc;
                // the low-pass disc's extent on the strip, widened like the ellipse's
                float da = 1.0f, db = 0.0f;
                if (LP) {
                    const float Yn = Ya > 0.0f ? Ya : (Yb < 0.0f ? Yb : 0.0f);
                    const bool in = Yn * Yn <= rd2 * 1.001f;
                    const float hw = sqrt_approx(fmaxf(rd2 * 1.001f - Yn * Yn, 0.0f)) + 0.05f;
                    const float lo = ceilf(xc - hw - 0.5f), hi = floorf(xc + hw - 0.5f);
                    da = in ? (lo < fx0 ? fx0 : (lo > fx1 ? fx1 + 1.0f : lo)) : 1.0f;
                    db = in ? (hi > fx1 ? fx1 : (hi < fx0 ? fx0 - 1.0f : hi)) : 0.0f;
                    if (!ell) {
                        keep = keep && da <= db;
                        ca = da;
                        cb = db;
                    }
                }
                float ext[2];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const float Y = Yt[side] < Ya ? Ya : Yb;
                    const float bb = B * Y + D;
                    const float cc = (Cc * Y + 2.0f * E) * Y + F;
                    const float sq = sqrt_approx(fmaxf(bb * bb - A * cc, 0.0f));
                    const float root = (side == 0 ? -bb - sq : -bb + sq) * iA;
                    ext[side] = Yt[side] >= Ya && Yt[side] <= Yb ? Xs[side] : root;
                }
                if (ell) {
                    // comparisons are false for NaN: a degenerate extent restricts nothing
                    const float lo = ceilf(ext[0] + xc - 0.5f - margin), hi = floorf(ext[1] + xc - 0.5f + margin);
                    ca = lo > ca ? (lo > cb ? cb + 1.0f : lo) : ca;
                    cb = hi < cb ? (hi < ca ? ca - 1.0f : hi) : cb;
                    if (da <= db) {
                        const bool empty = ca > cb;
                        ca = empty ? da : fminf(ca, da);
                        cb = empty ? db : fmaxf(cb, db);
                    }
                }
                keep = keep && ca <= cb;
            }
            // the 8-pixel block columns that [ca, cb] meets
            uint32_t bits = 0u;
#pragma unroll
            for (int bx = 0; bx < 4; ++bx) {
                const float c0 = ftx + 8.0f * (float)bx;
                bits |= (bx < WX && ca <= c0 + 7.0f && cb >= c0) ? (1u << bx) : 0u;
            }
            if (keep) m |= bits << (by * WX);
        }
    }
    return m;
}

// Next tile of a CTA: the tile at its own index (grid schedule) or at the
// head of a device work queue (persistent schedule) in the heavy-first tile
// order.  Contains __syncthreads in the persistent case, so it also
// separates consecutive tiles' use of shared memory.
__device__ __forceinline__ int next_tile_q(int persistent, uint32_t* queue, int* s_tile, bool first,
                                           const Cams& cams) {
    int i;
    if (!persistent) {
        i = first ? (int)blockIdx.x : INT_MAX;
    } else {
        __syncthreads();
        if (threadIdx.x == 0) *s_tile = (int)atomicAdd(queue, 1u);
        __syncthreads();
        i = *s_tile;
    }
    // the i-th tile of the heavy-first order
    return i < cams.total_tiles ? (cams.tile_order ? cams.tile_order[i] : i) : INT_MAX;
}

// exclusive scan of v[0, n) in shared memory by the whole CTA (n <= 8 *
// blockDim.x, blockDim.x a multiple of 32, <= 1024); returns the total.
// `red` is a 33-int shared scratch.  Contains __syncthreads.
__device__ __forceinline__ int block_exscan(int* v, int n, int* red) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    int loc[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = tid * per + k;
        loc[k] = (k < per && i < n) ? v[i] : 0;
        sum += loc[k];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) red[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < nw ? red[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) red[lane] = wi - w;
        if (lane == 31) red[32] = wi;
    }
    __syncthreads();
    int run = red[wid] + incl - sum;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = tid * per + k;
        if (k < per && i < n) { v[i] = run; run += loc[k]; }
    }
    const int total = red[32];
    __syncthreads();
    return total;
}

// block_exscan of v[i] | (v[i] != 0): the values' low bit also counts the
// nonzero entries (for counts kept in the high bits)
__device__ __forceinline__ int block_exscan_marked(int* v, int n, int* red) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    int loc[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = tid * per + k;
        loc[k] = (k < per && i < n) ? (v[i] | (v[i] != 0 ? 1 : 0)) : 0;
        sum += loc[k];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) red[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < nw ? red[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) red[lane] = wi - w;
        if (lane == 31) red[32] = wi;
    }
    __syncthreads();
    int run = red[wid] + incl - sum;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = tid * per + k;
        if (k < per && i < n) { v[i] = run; run += loc[k]; }
    }
    const int total = red[32];
    __syncthreads();
    return total;
}

__device__ __forceinline__ void warp_count(uint64_t* ctr, uint32_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(ctr), (unsigned long long)v);
}

// vector reduction into global memory (sm_90+): four floats, one request
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Order-preserving 64-bit key of (value, channel) for an argmax by integer
// maximum: larger values first, then smaller channel indices.
__device__ __forceinline__ unsigned long long argmax_key(float v, int c) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((unsigned long long)o << 32) | (0xFFFFFFFFu - (uint32_t)c);
}
__device__ __forceinline__ int argmax_channel(unsigned long long key) {
    return (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
}

// Launch of a render kernel over the tiles (one CTA per tile, or one resident
// wave for the persistent schedule), recording the measurement hook after it.
template <typename KernelT>
inline cudaError_t launch_tiles(KernelT kern, int threads, size_t smem, const Cams& cams, const RParams& P, const FwdArgs& a,
                               const AuxOut& x, int num_sms, cudaStream_t stream) {
    cudaError_t e = cudaSuccess;
    if (smem + 2048 > 48 * 1024) {  // above the default limit with the kernels' static shared memory (< 2 KB)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int grid = cams.total_tiles;
    if (a.persistent) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e != cudaSuccess) return e;
        grid = std::min(cams.total_tiles, max(1, per_sm) * num_sms);
    }
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, threads, smem, stream>>>(cams, P, a, x);
    e = cudaGetLastError();
    if (e == cudaSuccess) kernel_mark(stream);
    return e;
}


}  // namespace fss
