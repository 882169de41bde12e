// Projection and Precise Tile Intersection binning (Sec. 3.2) for sm_103a.
//
// k_project   one thread per (view, surfel) item: homogeneous transform T,
//             its adjugate about the projected centre, opacity-aware cutoff,
//             screen conic, SnugBox pixel range; appends visible items to a
//             compact list (unbounded conics to a per-view list instead).
//             Also counts each item's tiles (AccuTile per-row or per-column
//             intervals) into per-tile counters.
// k_emit      computes the double-float render records; one of its CTAs
//             scans the per-tile counts (tile ranges, total pairs, capacity,
//             the heavy-first tile order) while the others build records;
//             then writes each item into a slot of each of its tiles (slot
//             order is arbitrary; the per-tile sort restores a total order).
//
// Every tile decision is taken in binary32 with the fixed operation order
// that the FP64 checker's binning mirror also follows, so tile lists compare
// bit for bit.  This translation unit is compiled with -fmad=false and
// spells each rounding with an _rn intrinsic, so no multiply-add is fused.
#include "fss_internal.cuh"
#include "kernels.cuh"

namespace fss {

namespace {

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fq(float a) { return __fsqrt_rn(a); }

// frexpf and ldexpf for the chain below, from the binary32 layout: for a
// normal x > 0, x = m 2^e with m in [1/2, 1) takes the exponent field and
// the mantissa bits; x 2^k (one rounding, as ldexpf) is a multiply by the
// exact power of two whenever 2^k is a normal number.  Other cases (zero,
// subnormal, non-finite, exponents out of that range) call the library.
__device__ __forceinline__ float frexp32(float x, int* e) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t be = (b >> 23) & 0xffu;
    if (be == 0u || be == 0xffu || (b >> 31)) return frexpf(x, e);
    *e = (int)be - 126;
    return __uint_as_float((b & 0x807fffffu) | 0x3f000000u);
}
__device__ __forceinline__ float ldexp32(float x, int k) {
    if (k < -126 || k > 127) return ldexpf(x, k);
    return __fmul_rn(x, __uint_as_float((uint32_t)(k + 127) << 23));
}

// natural logarithm of x > 0 in binary32, the same operation sequence as the
// checker's binning mirror: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
// ln m = 2 atanh(s), s = (m - 1)/(m + 1), series to s^9 (|s| <= 0.1716).
__device__ __forceinline__ float ln32(float x) {
    int e;
    float m = frexp32(x, &e);
    if (m < 0.70710677f) { m = fm(m, 2.0f); e = e - 1; }
    const float s = fdv(fs(m, 1.0f), fa(m, 1.0f));
    const float s2 = fm(s, s);
    float p = fm(s2, 1.0f / 9.0f);
    p = fm(fa(p, 1.0f / 7.0f), s2);
    p = fm(fa(p, 1.0f / 5.0f), s2);
    p = fm(fa(p, 1.0f / 3.0f), s2);
    p = fa(p, 1.0f);
    return fa(fm((float)e, 0.6931472f), fm(fm(2.0f, s), p));
}

// ---- double-float arithmetic (hi + lo, ~48 significant bits) ----------------
// Error-free sums (Knuth's two-sum, 6 operations) and products (the exact
// low part of a*b from one fused multiply-add), renormalised after every
// operation.  Used only for the per-surfel render record, whose ray-splat
// homography is ill-conditioned for surfels seen close to edge-on.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = fa(a, b), bb = fs(s, a);
    return {s, fa(fs(a, fs(s, bb)), fs(b, bb))};
}
__device__ __forceinline__ df quick_two_sum(float s, float e) {
    const float h = fa(s, e);
    return {h, fs(e, fs(h, s))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = fm(a, b);
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df dadd(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, fa(s.lo, fa(x.lo, y.lo)));
}
__device__ __forceinline__ df dneg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df dsub(df x, df y) { return dadd(x, dneg(y)); }
__device__ __forceinline__ df dmul(df x, df y) {
    const df p = two_prod(x.hi, y.hi);
    return quick_two_sum(p.hi, fa(p.lo, fa(fm(x.hi, y.lo), fm(x.lo, y.hi))));
}
__device__ __forceinline__ df dmulf(df x, float f) {
    const df p = two_prod(x.hi, f);
    return quick_two_sum(p.hi, fa(p.lo, fm(x.lo, f)));
}
__device__ __forceinline__ df dfrom(float a) { return {a, 0.0f}; }
// (R v)_r with binary32 R and double-float v
__device__ __forceinline__ void dmvec(const float* R, const df v[3], df o[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) o[r] = dadd(dadd(dmulf(v[0], R[3 * r]), dmulf(v[1], R[3 * r + 1])), dmulf(v[2], R[3 * r + 2]));
}
__device__ __forceinline__ void dcross(const df a[3], const df b[3], df o[3]) {
    o[0] = dsub(dmul(a[1], b[2]), dmul(a[2], b[1]));
    o[1] = dsub(dmul(a[2], b[0]), dmul(a[0], b[2]));
    o[2] = dsub(dmul(a[0], b[1]), dmul(a[1], b[0]));
}

// (R v)_r = (R_r0 v0 + R_r1 v1) + R_r2 v2
__device__ __forceinline__ void mvec(const float* R, const float v[3], float o[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) o[r] = fa(fa(fm(R[3 * r], v[0]), fm(R[3 * r + 1], v[1])), fm(R[3 * r + 2], v[2]));
}

__device__ __forceinline__ void crossf(const float a[3], const float b[3], float o[3]) {
    o[0] = fs(fm(a[1], b[2]), fm(a[2], b[1]));
    o[1] = fs(fm(a[2], b[0]), fm(a[0], b[2]));
    o[2] = fs(fm(a[0], b[1]), fm(a[1], b[0]));
}

// Q_ab = (m0_a m0_b + m1_a m1_b) - kk (m2_a m2_b), (A,B,C,D,E,F) = (Q00,Q01,Q11,Q02,Q12,Q22)
__device__ __forceinline__ void conic(const float m[9], float kk, float q[6]) {
    const int ia[6] = {0, 0, 1, 0, 1, 2}, ib[6] = {0, 1, 1, 2, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int a = ia[k], b = ib[k];
        const float s = fa(fm(m[a], m[b]), fm(m[3 + a], m[3 + b]));
        const float t = fm(kk, fm(m[6 + a], m[6 + b]));
        q[k] = fs(s, t);
    }
}

// centre and half extents of the ellipse q <= 0; false if it is empty
__device__ __forceinline__ bool ellipse(const float q[6], float& X0, float& Y0, float& hx, float& hy) {
    const float A = q[0], B = q[1], C = q[2], D = q[3], E = q[4], F = q[5];
    const float g = fs(fm(A, C), fm(B, B));
    X0 = fdv(fs(fm(B, E), fm(C, D)), g);
    Y0 = fdv(fs(fm(B, D), fm(A, E)), g);
    const float Fp = fa(fa(F, fm(D, X0)), fm(E, Y0));
    if (!(Fp < 0.0f)) return false;
    const float nF = -Fp;
    hx = fq(fdv(fm(nF, C), g));
    hy = fq(fdv(fm(nF, A), g));
    return true;
}

// pixel indices whose centres lie in [lo + 0.5, hi + 0.5], clipped to [0, n-1]
__device__ __forceinline__ bool pix_range(float lo, float hi, int n, int& a, int& b) {
    const float fl = ceilf(lo), fh = floorf(hi);
    if (!(fl <= fh)) return false;
    if (fh < 0.0f || fl > (float)(n - 1)) return false;
    a = fl < 0.0f ? 0 : (int)fl;
    b = fh > (float)(n - 1) ? n - 1 : (int)fh;
    return a <= b;
}

// S20b: pixel interval [a, b] (clipped to [lo_clip, hi_clip]) of the
// low-pass screen disc of radius^2 rd2 about the local origin on the strip
// [Sa, Sb] of the other coordinate; a > b when it misses the strip
__device__ __forceinline__ void disc_strip(float rd2, float Sa, float Sb, float origin, int lo_clip, int hi_clip,
                                           int& a, int& b) {
    a = 1;
    b = 0;
    const float Sn = Sa > 0.0f ? Sa : (Sb < 0.0f ? Sb : 0.0f);
    const float s2 = fm(Sn, Sn);
    if (!(s2 <= rd2)) return;
    const float hw = fq(fs(rd2, s2));
    const float fl = ceilf(fs(fa(-hw, origin), 0.5f)), fh = floorf(fs(fa(hw, origin), 0.5f));
    if (!(fl <= fh) || fh < (float)lo_clip || fl > (float)hi_clip) return;
    a = fl < (float)lo_clip ? lo_clip : (int)fl;
    b = fh > (float)hi_clip ? hi_clip : (int)fh;
}

// union of an ellipse interval [a, b] (empty if a > b) with a disc interval
__device__ __forceinline__ void hull_interval(int& a, int& b, int da, int db) {
    if (da > db) return;
    if (a > b) { a = da; b = db; return; }
    a = min(a, da);
    b = max(b, db);
}

// AccuTile: the inner tile interval of one outer tile line (a row of tiles
// when `rows`, else a column).  On a row strip [Ya, Yb] (local coordinates)
// the ellipse's extreme abscissae are its left/right tangent points when
// these fall inside the strip, else the roots of
//   A x^2 + 2(B y + D) x + (C y^2 + 2 E y + F) = 0
// at the nearer strip edge.  A column is the same with x and y exchanged
// (A <-> C, D <-> E, and the centre, half extents and pixel ranges), so one
// code path serves both, its operands picked by selects; both candidates of
// each side are computed and one is selected.  The lanes of a warp,
// holding different items and line kinds, then never split on these
// branches (a divergent version measured ~1800 cycles per call).
__device__ __forceinline__ bool accu_line(const BinRec& r, bool rows, int ts, int o, int& ta, int& tb) {
    const float A = rows ? r.A : r.C, C = rows ? r.C : r.A, D = rows ? r.D : r.E, E = rows ? r.E : r.D;
    const float X0 = rows ? r.X0 : r.Y0, hx = rows ? r.hx : r.hy;
    const float xc = rows ? r.xc : r.yc, yc = rows ? r.yc : r.xc;
    const int p0 = rows ? r.px0 : r.py0, p1 = rows ? r.px1 : r.py1;  // inner pixel range
    const int q0 = rows ? r.py0 : r.px0, q1 = rows ? r.py1 : r.px1;  // outer pixel range
    const int ra = max(o * ts, q0), rb = min(o * ts + ts - 1, q1);
    if (ra > rb) return false;
    const float Ya = fs(fa((float)ra, 0.5f), yc), Yb = fs(fa((float)rb, 0.5f), yc);
    int da = 1, db = 0;  // S20b
    if (r.flags & BR_LOWPASS) disc_strip(r.rd2, Ya, Yb, xc, p0, p1, da, db);
    if (!(r.flags & BR_ELL)) {
        if (da > db) return false;
        ta = da >> (__ffs(ts) - 1);
        tb = db >> (__ffs(ts) - 1);
        return true;
    }
    float ext[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const float Xs = side == 0 ? fs(X0, hx) : fa(X0, hx);
        const float t = fa(fm(r.B, Xs), E);
        const float Yt = fdv(-t, C);
        const bool tangent = Yt >= Ya && Yt <= Yb;
        const float Y = Yt < Ya ? Ya : Yb;
        const float bb = fa(fm(r.B, Y), D);
        const float cc = fa(fa(fm(fm(C, Y), Y), fm(fm(2.0f, E), Y)), r.F);
        float disc = fs(fm(bb, bb), fm(A, cc));
        disc = disc < 0.0f ? 0.0f : disc;
        const float sq = fq(disc), nb = -bb;
        const float root = fdv(side == 0 ? fs(nb, sq) : fa(nb, sq), A);
        ext[side] = tangent ? Xs : root;
    }
    const float fl = ceilf(fs(fa(ext[0], xc), 0.5f)), fh = floorf(fs(fa(ext[1], xc), 0.5f));
    const bool hit = fl <= fh && !(fh < (float)p0 || fl > (float)p1);
    int a = hit ? (fl < (float)p0 ? p0 : (int)fl) : 1;
    int b = hit ? (fh > (float)p1 ? p1 : (int)fh) : 0;
    hull_interval(a, b, da, db);
    if (a > b) return false;
    ta = a >> (__ffs(ts) - 1);
    tb = b >> (__ffs(ts) - 1);
    return true;
}

// Outer lines of an item's tile set: rows if the tile span in y does not
// exceed the span in x (or for the box modes), else columns (SnugBox's
// traversal over the smaller span).
struct Lines {
    int n;          // number of outer lines
    int first;      // first outer coordinate
    bool rows;      // outer loop over tile rows
    bool accurate;  // per-line AccuTile interval (else the full rectangle)
};

__device__ __forceinline__ Lines lines_of(const BinRec& r, int bin_mode) {
    Lines L;
    const int xs = r.tx1 - r.tx0 + 1, ys = r.ty1 - r.ty0 + 1;
    L.accurate = bin_mode == FSS_BIN_ACCU;
    L.rows = !L.accurate || ys <= xs;
    L.n = L.rows ? ys : xs;
    L.first = L.rows ? r.ty0 : r.tx0;
    return L;
}

// inner tile interval [a, b] of outer line `o` (an absolute tile row/column)
__device__ __forceinline__ bool line_interval(const BinRec& r, const Lines& L, int ts, int o, int& a, int& b) {
    if (!L.accurate) {
        a = L.rows ? r.tx0 : r.ty0;
        b = L.rows ? r.tx1 : r.ty1;
        return true;
    }
    return accu_line(r, L.rows, ts, o, a, b);
}

// view of item (items are view-major, view * N + surfel, < 2^32)
__device__ __forceinline__ int view_of_item(int64_t item, int64_t N) {
    return N >= ((int64_t)1 << 32) || item < N ? 0 : (int)((uint32_t)item / (uint32_t)N);
}

// Tile work of a warp's items spread over its lanes.  The outer lines of
// the 32 lanes' items are numbered in lane order ((lane, line) units) and
// taken 32 at a time, one per lane, so that an item with many lines no
// longer runs them one after another in its own lane while the others wait.
// The warp's slices of shared memory hold each lane's binning record and
// item, and the inclusive prefix of the line counts.
struct WarpLines {
    BinRec* br;      // [32]
    uint32_t* item;  // [32]
    int* pre;        // [32]
};

// every lane of the warp calls this with its own line count (0 for no
// item) after writing its record and item; returns the warp's total
__device__ __forceinline__ int warp_line_prefix(const WarpLines& w, int nl) {
    const int lane = threadIdx.x & 31;
    int incl = nl;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    w.pre[lane] = incl;
    __syncwarp();
    return __shfl_sync(0xffffffffu, incl, 31);
}

// g(owner lane, item, camera, rows, outer line, first tile, last tile) for
// every non-empty line interval of the warp's items (inner tiles a..b)
template <typename G>
__device__ __forceinline__ void warp_lines(const Cams& cams, const RParams& P, const WarpLines& w, int total, G&& g) {
    const int lane = threadIdx.x & 31;
    for (int u = lane; u < total; u += 32) {
        int j = 0;  // owner: the first lane whose inclusive prefix exceeds u
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) j += w.pre[j + step - 1] <= u ? step : 0;
        const BinRec r = w.br[j];
        const Lines L = lines_of(r, P.bin_mode);
        const int o = L.first + (u - (w.pre[j] - L.n));
        int a, b;
        if (!line_interval(r, L, P.ts, o, a, b)) continue;
        const uint32_t item = w.item[j];
        g(j, item, cams.c[view_of_item(item, P.N)], L.rows, o, a, b);
    }
}

}  // namespace

// S3 (centre), S4 (near plane), S5 (opacity) and S5b (conservative frustum
// test): the cheap culls, which remove most surfels of a view before the
// rest of the chain.  Returns false when the item is culled; pc and o as
// computed (o = 0 if the depth test failed first).
// the surfel inputs the culls read, loaded together so that their latencies overlap
struct CullIn {
    float pm[3];
    float o;
    float2 sc;
};
__device__ __forceinline__ CullIn load_cull_in(const float* __restrict__ means, const float* __restrict__ scales,
                                               const float* __restrict__ opac, int64_t s) {
    CullIn c;
    c.pm[0] = __ldg(means + 3 * s);
    c.pm[1] = __ldg(means + 3 * s + 1);
    c.pm[2] = __ldg(means + 3 * s + 2);
    c.o = __ldg(opac + s);
    c.sc = __ldg(reinterpret_cast<const float2*>(scales) + s);
    return c;
}

__device__ __forceinline__ bool early_culls(const CamDev& cam, const RParams& P, const CullIn& in, float pc[3],
                                            float& o) {
    float e[3];
    mvec(cam.R, in.pm, e);
#pragma unroll
    for (int i = 0; i < 3; ++i) pc[i] = fa(e[i], cam.t[i]);
    o = 0.0f;
    if (!(pc[2] > cam.near_plane)) return false;
    // S5
    o = in.o;
    if (!(o >= P.alpha_min)) return false;
    // S5b: the binning disk lies in the sphere of radius
    // rho = sqrt(k^2 (1 + 2^-10)) max(r_u, r_v) about the centre; if that
    // sphere is in front of the camera and its projection's bounding box
    // misses every pixel centre by more than a pixel, no pixel can be reached.
    const float2 scp = in.sc;
    const float kk = fm(fm(2.0f, ln32(fdv(o, P.alpha_min))), 1.0009765625f);
    const float rho = fa(fm(fm(fq(fmaxf(kk, 0.0f)), fmaxf(scp.x, scp.y)), 1.001f), 1e-6f);
    const float zlo = fs(pc[2], rho), zhi = fa(pc[2], rho);
    if (zlo > 0.0f) {
        const float xa = fs(pc[0], rho), xb = fa(pc[0], rho), ya = fs(pc[1], rho), yb = fa(pc[1], rho);
        // extremes of x/z and y/z over the box [xa, xb] x [ya, yb] x [zlo, zhi]
        const float uxmax = fdv(xb, xb >= 0.0f ? zlo : zhi), uxmin = fdv(xa, xa >= 0.0f ? zhi : zlo);
        const float uymax = fdv(yb, yb >= 0.0f ? zlo : zhi), uymin = fdv(ya, ya >= 0.0f ? zhi : zlo);
        const float pxmax = fa(fm(cam.fx, uxmax), cam.cx), pxmin = fa(fm(cam.fx, uxmin), cam.cx);
        const float pymax = fa(fm(cam.fy, uymax), cam.cy), pymin = fa(fm(cam.fy, uymin), cam.cy);
        // S5b': the low-pass filter's screen disc widens the margins
        const float mg = P.lowpass ? fa(0.5f, fq(fm(fmaxf(kk, 0.0f), 0.5f))) : 0.5f;
        if (pxmax < -mg || pxmin > fa((float)cam.W, mg) || pymax < -mg || pymin > fa((float)cam.H, mg))
            return false;
    }
    return true;
}

constexpr int PROJ_ITEMS = 1024;  // items per CTA of k_project
constexpr int PROJ_THREADS = 256;

// ---------------------------------------------------------------------------
// k_project: (view, surfel) items, PROJ_ITEMS per CTA
//
// Stage A runs the cheap culls (depth, opacity, frustum) one thread per item
// and queues the survivors in shared memory; stage B runs the rest of the
// chain one thread per survivor, so the few visible surfels of a view fill
// whole warps instead of one lane in each.  A visible item with a bounded conic counts
// its tiles (fire-and-forget adds into the per-tile counters, cleared by the
// host call before this kernel) and is appended to the narrow list, or to
// the wide list when it spans more than WIDE_TILES tiles; an unbounded item
// goes to its view's list instead (every tile of the view includes it).
// Appends and gradient-slot claims are aggregated per warp.
// ---------------------------------------------------------------------------
constexpr uint32_t WIDE_TILES = 32;

__global__ void __launch_bounds__(PROJ_THREADS, 4) k_project(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                                 const float* __restrict__ means, const float* __restrict__ scales,
                                                 const float* __restrict__ quats, const float* __restrict__ opac,
                                                 float4* __restrict__ rec, BinRec* __restrict__ binrec,
                                                 uint32_t* __restrict__ count, uint32_t* __restrict__ tile_cnt,
                                                 uint32_t* __restrict__ vis_list, uint32_t* __restrict__ wide_list,
                                                 uint32_t* __restrict__ unb_list, int32_t* __restrict__ splat_slot,
                                                 int32_t* __restrict__ slot_surf, Status* __restrict__ st) {
    __shared__ uint32_t s_q[PROJ_ITEMS];
    __shared__ int s_nq;
    __shared__ BinRec s_br[PROJ_THREADS];
    __shared__ uint32_t s_item[PROJ_THREADS], s_cnt[PROJ_THREADS];
    __shared__ int s_pre[PROJ_THREADS];
    const int wb = threadIdx.x & ~31;
    const WarpLines wl{s_br + wb, s_item + wb, s_pre + wb};
    if (st->err) return;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_nq = 0;
    __syncthreads();
    // stage A: the cheap culls for PROJ_ITEMS items (each thread's items loaded
    // together first); survivors queued in shared memory
    const int64_t base = (int64_t)blockIdx.x * PROJ_ITEMS;
    constexpr int PER = PROJ_ITEMS / PROJ_THREADS;
    CullIn in[PER];
    int vw[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int64_t it = base + threadIdx.x + i * PROJ_THREADS;
        vw[i] = 0;
        if (it < P.n_items) {
            vw[i] = view_of_item(it, P.N);
            in[i] = load_cull_in(means, scales, opac, it - (int64_t)vw[i] * P.N);
        }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int k = threadIdx.x + i * PROJ_THREADS;
        const int64_t it = base + k;
        bool keep = false;
        if (it < P.n_items) {
            float pc[3], o;
            keep = early_culls(cams.c[vw[i]], P, in[i], pc, o);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        int b = 0;
        if (lane == 0 && m) b = atomicAdd(&s_nq, __popc(m));
        b = __shfl_sync(0xffffffffu, b, 0);
        if (keep) s_q[b + __popc(m & ((1u << lane) - 1u))] = (uint32_t)k;
    }
    __syncthreads();
    const int nq = s_nq;
    // stage B: the whole chain for the survivors, packed densely into warps
    // (warp-uniform loop: the appends below use whole-warp ballots)
    for (int q0 = threadIdx.x & ~31; q0 < nq; q0 += blockDim.x) {
    const int64_t item = q0 + lane < nq ? base + s_q[q0 + lane] : P.n_items;
    bool vis = false, wide = false, unb = false, claim = false;
    int64_t claim_s = 0;
    int view = 0;
    BinRec br;
    if (item < P.n_items) {
        view = view_of_item(item, P.N);
        const int64_t s = item - (int64_t)view * P.N;
        const CamDev& cam = cams.c[view];
        br.flags = 0;
        br.px0 = br.py0 = br.tx0 = br.ty0 = 1;
        br.px1 = br.py1 = br.tx1 = br.ty1 = 0;
        br.A = br.B = br.C = br.D = br.E = br.F = 0.0f;
        br.X0 = br.Y0 = br.hx = br.hy = br.xc = br.yc = 0.0f;
        br.rd2 = 0.0f;
        br.pad[0] = br.pad[1] = 0;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
        do {
            // S3 (centre), S4, S5, S5b first: the order of the cull tests does not change the result
            // (the rotation is loaded beside the cull inputs, so that the latencies overlap)
            const CullIn ci = load_cull_in(means, scales, opac, s);
            const float4 q4 = __ldg(reinterpret_cast<const float4*>(quats) + s);
            float pc[3], o;
            const bool pass = early_culls(cam, P, ci, pc, o);
            r3.y = pc[2];
            r3.x = o;
            if (!pass) break;
            // S1
            const float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
            const float n2 = fa(fa(fa(fm(qw, qw), fm(qx, qx)), fm(qy, qy)), fm(qz, qz));
            if (!(n2 > 0.0f)) break;
            const float nn = fq(n2);
            const float w = fdv(qw, nn), x = fdv(qx, nn), y = fdv(qy, nn), z = fdv(qz, nn);
            // S2
            float tu[3], tv[3];
            tu[0] = fs(1.0f, fm(2.0f, fa(fm(y, y), fm(z, z))));
            tu[1] = fm(2.0f, fa(fm(x, y), fm(w, z)));
            tu[2] = fm(2.0f, fs(fm(x, z), fm(w, y)));
            tv[0] = fm(2.0f, fs(fm(x, y), fm(w, z)));
            tv[1] = fs(1.0f, fm(2.0f, fa(fm(x, x), fm(z, z))));
            tv[2] = fm(2.0f, fa(fm(y, z), fm(w, x)));
            // S3 (tangent columns)
            const float su = ci.sc.x, sv = ci.sc.y;
            float au[3], av[3], e[3];
            mvec(cam.R, tu, e);
#pragma unroll
            for (int i = 0; i < 3; ++i) au[i] = fm(su, e[i]);
            mvec(cam.R, tv, e);
#pragma unroll
            for (int i = 0; i < 3; ++i) av[i] = fm(sv, e[i]);
            // S6: k^2 = 2 ln(o / alpha_min)
            const float k2 = fm(2.0f, ln32(fdv(o, P.alpha_min)));
            r3.z = k2;
            // S7
            float c[3][3];
            const float* src[3] = {au, av, pc};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                c[j][0] = fa(fm(cam.fx, src[j][0]), fm(cam.cx, src[j][2]));
                c[j][1] = fa(fm(cam.fy, src[j][1]), fm(cam.cy, src[j][2]));
                c[j][2] = src[j][2];
            }
            // S8
            const float xc = fdv(c[2][0], c[2][2]);
            const float yc = fdv(c[2][1], c[2][2]);
            // S9
            float d[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                d[j][0] = fs(c[j][0], fm(xc, c[j][2]));
                d[j][1] = fs(c[j][1], fm(yc, c[j][2]));
                d[j][2] = c[j][2];
            }
            // S10
            float m[9];
            crossf(d[1], d[2], &m[0]);
            crossf(d[2], d[0], &m[3]);
            crossf(d[0], d[1], &m[6]);
            // S11
            float det = fa(fa(fm(d[0][0], m[0]), fm(d[0][1], m[1])), fm(d[0][2], m[2]));
            // S12: edge-on cull
            const float pn = fq(fa(fa(fm(pc[0], pc[0]), fm(pc[1], pc[1])), fm(pc[2], pc[2])));
            const float lim = fm(1e-3f, fm(fm(fm(fm(cam.fx, cam.fy), su), sv), pn));
            if (!(fabsf(det) > lim)) break;
            // S13: exact power-of-two rescale
            float mx = 0.0f;
#pragma unroll
            for (int i = 0; i < 9; ++i) mx = fabsf(m[i]) > mx ? fabsf(m[i]) : mx;
            if (!(mx > 0.0f)) break;
            int ex;
            frexp32(mx, &ex);
#pragma unroll
            for (int i = 0; i < 9; ++i) m[i] = ldexp32(m[i], -ex);
            det = ldexp32(det, -ex);
            r3.w = ldexp32(1.0f, -ex);
            r0 = make_float4(m[0], m[1], m[2], xc);
            r1 = make_float4(m[3], m[4], m[5], yc);
            r2 = make_float4(m[6], m[7], m[8], det);
            br.xc = xc;
            br.yc = yc;
            // S14
            const float kb = fm(k2, 1.0009765625f);
            float q[6];
            conic(m, kb, q);
            br.A = q[0]; br.B = q[1]; br.C = q[2]; br.D = q[3]; br.E = q[4]; br.F = q[5];
            int px0, px1, py0, py1;
            // S15
            const float g = fs(fm(q[0], q[2]), fm(q[1], q[1]));
            if (!(q[0] > 0.0f && g > 0.0f)) {
                br.flags |= BR_UNBOUNDED;
                px0 = 0; px1 = cam.W - 1; py0 = 0; py1 = cam.H - 1;
            } else {
                // S16, S17: the ellipse's pixel range
                int e0 = 0, e1 = 0, f0 = 0, f1 = 0;
                bool ell = ellipse(q, br.X0, br.Y0, br.hx, br.hy);
                if (ell)
                    ell = pix_range(fs(fa(fs(br.X0, br.hx), xc), 0.5f), fs(fa(fa(br.X0, br.hx), xc), 0.5f), cam.W, e0,
                                    e1) &&
                          pix_range(fs(fa(fs(br.Y0, br.hy), yc), 0.5f), fs(fa(fa(br.Y0, br.hy), yc), 0.5f), cam.H, f0,
                                    f1);
                // S17b: the low-pass screen disc's, then the union
                int g0 = 0, g1 = 0, h0 = 0, h1 = 0;
                bool disc = false;
                if (P.lowpass) {
                    br.flags |= BR_LOWPASS;
                    br.rd2 = fm(kb, 0.5f);
                    const float rd = fq(br.rd2);
                    disc = pix_range(fs(fs(xc, rd), 0.5f), fs(fa(xc, rd), 0.5f), cam.W, g0, g1) &&
                           pix_range(fs(fs(yc, rd), 0.5f), fs(fa(yc, rd), 0.5f), cam.H, h0, h1);
                }
                if (!ell && !disc) break;
                if (ell) br.flags |= BR_ELL;
                px0 = ell ? (disc ? min(e0, g0) : e0) : g0;
                px1 = ell ? (disc ? max(e1, g1) : e1) : g1;
                py0 = ell ? (disc ? min(f0, h0) : f0) : h0;
                py1 = ell ? (disc ? max(f1, h1) : f1) : h1;
            }
            br.flags |= BR_VISIBLE;
            br.px0 = (int16_t)px0; br.px1 = (int16_t)px1; br.py0 = (int16_t)py0; br.py1 = (int16_t)py1;
            // S18
            const int ts = P.ts;
            const int lts = __ffs(ts) - 1;  // tile sizes are powers of two; pixel indices are >= 0
            int tx0 = px0 >> lts, tx1 = px1 >> lts, ty0 = py0 >> lts, ty1 = py1 >> lts;
            // S19
            if (P.bin_mode == FSS_BIN_AABB && !(br.flags & BR_UNBOUNDED)) {
                float k2a = fm(2.0f, ln32(fdv(1.0f, P.alpha_min)));
                if (kb > k2a) k2a = kb;
                float qa[6], X0, Y0, hx, hy;
                conic(m, k2a, qa);
                const float ga = fs(fm(qa[0], qa[2]), fm(qa[1], qa[1]));
                int ax0 = 0, ax1 = cam.W - 1, ay0 = 0, ay1 = cam.H - 1;
                if (qa[0] > 0.0f && ga > 0.0f && ellipse(qa, X0, Y0, hx, hy)) {
                    const float h = hx > hy ? hx : hy;
                    if (!pix_range(fs(fa(fs(X0, h), xc), 0.5f), fs(fa(fa(X0, h), xc), 0.5f), cam.W, ax0, ax1)) {
                        ax0 = px0; ax1 = px1;
                    }
                    if (!pix_range(fs(fa(fs(Y0, h), yc), 0.5f), fs(fa(fa(Y0, h), yc), 0.5f), cam.H, ay0, ay1)) {
                        ay0 = py0; ay1 = py1;
                    }
                }
                ax0 = min(ax0, px0); ax1 = max(ax1, px1);
                ay0 = min(ay0, py0); ay1 = max(ay1, py1);
                tx0 = ax0 >> lts; tx1 = ax1 >> lts; ty0 = ay0 >> lts; ty1 = ay1 >> lts;
            }
            br.tx0 = (int16_t)tx0; br.tx1 = (int16_t)tx1; br.ty0 = (int16_t)ty0; br.ty1 = (int16_t)ty1;
        } while (0);
        vis = (br.flags & BR_VISIBLE) && !(br.flags & BR_UNBOUNDED);
        unb = (br.flags & BR_VISIBLE) && (br.flags & BR_UNBOUNDED);
        if (vis || unb) {  // records of culled items are never read
            float4* rr = rec + 4 * item;
            rr[0] = r0; rr[1] = r1; rr[2] = r2; rr[3] = r3;
            binrec[item] = br;
            // one gradient slot per surfel visible in any view (-1 -> -2 claims it);
            // with one view every item is a distinct surfel, so no round trip
            claim = cams.n == 1 || atomicCAS(&splat_slot[s], -1, -2) == -1;
            claim_s = s;
        }
    }
    // per-tile pair counts (S20 intervals), the warp's lines spread over its lanes
    {
        const int lane = threadIdx.x & 31;
        if (vis) wl.br[lane] = br;
        wl.item[lane] = (uint32_t)item;
        s_cnt[threadIdx.x] = 0u;
        const int total = warp_line_prefix(wl, vis ? lines_of(br, P.bin_mode).n : 0);
        warp_lines(cams, P, wl, total, [&](int j, uint32_t, const CamDev& cam, bool rows, int o, int a, int b) {
            for (int k = a; k <= b; ++k) {
                const int tx = rows ? k : o, ty = rows ? o : k;
                const int tt = cam.tile_off + ty * cam.tiles_x + tx;
                if (in_bounds(st, SITE_TILE, tt, cams.total_tiles)) atomicAdd(&tile_cnt[(size_t)tt * TC_STRIDE], 1u);
            }
            atomicAdd(&s_cnt[wb + j], (uint32_t)(b - a + 1));
        });
        __syncwarp();
        if (vis) {
            const uint32_t cnt = s_cnt[threadIdx.x];
            count[item] = cnt;
            wide = cnt > WIDE_TILES;
        }
        __syncwarp();  // the slices are reused by the warp's next survivors
    }
    // warp-aggregated appends (one global atomic per warp and counter, no CTA barrier)
    {
        const int lane = threadIdx.x & 31;
        const unsigned lt = (1u << lane) - 1u;
        const bool narrow = vis && !wide, wid = vis && wide;
        const unsigned mn = __ballot_sync(0xffffffffu, narrow), mw = __ballot_sync(0xffffffffu, wid);
        const unsigned mc = __ballot_sync(0xffffffffu, claim);
        uint32_t bn = 0, bw = 0, bc = 0;
        if (lane == 0) {
            if (mn) bn = atomicAdd(&st->nvis, (uint32_t)__popc(mn));
            if (mw) bw = atomicAdd(&st->nwide, (uint32_t)__popc(mw));
            if (mc) bc = atomicAdd(&st->nslot, (uint32_t)__popc(mc));
        }
        bn = __shfl_sync(0xffffffffu, bn, 0);
        bw = __shfl_sync(0xffffffffu, bw, 0);
        bc = __shfl_sync(0xffffffffu, bc, 0);
        if (narrow && in_bounds(st, SITE_VIS_LIST, bn + __popc(mn & lt), P.n_items))
            vis_list[bn + __popc(mn & lt)] = (uint32_t)item;
        if (wid && in_bounds(st, SITE_VIS_LIST, bw + __popc(mw & lt), P.n_items))
            wide_list[bw + __popc(mw & lt)] = (uint32_t)item;
        if (claim) {
            const int32_t sl = (int32_t)(bc + __popc(mc & lt));
            if (in_bounds(st, SITE_SLOT, sl, P.N) && in_bounds(st, SITE_SLOT, claim_s, P.N)) {
                splat_slot[claim_s] = sl;
                slot_surf[sl] = (int32_t)claim_s;
            }
        }
    }
    if (unb) {
        const uint32_t k = atomicAdd(&st->unb_cnt[view], 1u);
        if (in_bounds(st, SITE_VIS_LIST, k, P.N)) unb_list[(int64_t)view * P.N + k] = (uint32_t)item;
    }
    }  // survivors
}

// ---------------------------------------------------------------------------
// Tile scan, run by one CTA of k_emit (any block size, a multiple of 32):
// per-tile totals (bounded pairs + the view's unbounded items) -> exclusive
// scan -> ranges; the tile counters become the emit cursors.  Then the
// heavy-first tile order: a counting sort of the tiles by pair count,
// descending, in buckets of 16 pairs (the order within a bucket is
// arbitrary).  The tile kernels take tiles in this order, so that the last
// tiles to start are light ones: the work per tile varies severalfold, and
// in index order a heavy tile starting late sets the kernel's end.
// ---------------------------------------------------------------------------
constexpr int ORDER_BUCKETS = 256;  // 32 lanes x 8
__device__ __forceinline__ int order_bucket(int2 r) { return min(ORDER_BUCKETS - 1, (r.y - r.x) >> 4); }

__device__ void scan_tiles(const Cams& cams, const RParams& P, uint32_t* __restrict__ tile_cnt,
                           int2* __restrict__ ranges, Status* __restrict__ st) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nt = cams.total_tiles;
    constexpr int ITEMS = 8;
    for (int base = 0; base < nt; base += blockDim.x * ITEMS) {
        uint32_t v[ITEMS];
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int t = base + threadIdx.x * ITEMS + k;
            v[k] = t < nt ? tile_cnt[(size_t)t * TC_STRIDE] + st->unb_cnt[view_of_tile(cams, t)] : 0u;
            sum += v[k];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t w = lane < nw ? warp_tot[lane] : 0u, wi = w;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, off);
                if (lane >= off) wi += y;
            }
            warp_tot[lane] = wi - w;  // exclusive
        }
        __syncthreads();
        uint64_t run = carry_s + warp_tot[wid] + (incl - sum);
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int t = base + threadIdx.x * ITEMS + k;
            if (t < nt) {
                const uint64_t s0 = run;
                run += v[k];
                const bool fits = run <= (uint64_t)P.pair_cap;
                ranges[t] = make_int2(fits ? (int)s0 : 0, fits ? (int)run : 0);
                tile_cnt[(size_t)t * TC_STRIDE] = fits ? (uint32_t)s0 : 0u;  // emit cursor
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry_s = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->pairs_needed = (int64_t)carry_s;
        if (carry_s > (uint64_t)P.pair_cap) atomicOr(&st->err, ERR_CAPACITY);
    }
}

// heavy-first order of the tiles from their ranges (a frame over capacity
// has empty ranges: any order)
__device__ void heavy_first_order(const Cams& cams, const int2* __restrict__ ranges, int32_t* __restrict__ order) {
    __shared__ uint32_t ord[ORDER_BUCKETS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nt = cams.total_tiles;
    for (int b = threadIdx.x; b < ORDER_BUCKETS; b += blockDim.x) ord[b] = 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) atomicAdd(&ord[order_bucket(ranges[t])], 1u);
    __syncthreads();
    if (wid == 0) {  // first position of each bucket, heaviest bucket first
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            c[k] = ord[ORDER_BUCKETS - 1 - (8 * lane + k)];
            sum += c[k];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            ord[ORDER_BUCKETS - 1 - (8 * lane + k)] = run;
            run += c[k];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) order[atomicAdd(&ord[order_bucket(ranges[t])], 1u)] = t;
}

// failure-detection test hook (fss_test_hold_scan): when set, the scanning
// CTA keeps its result to itself, so the other CTAs' bounded wait runs out
__device__ int g_hold_scan = 0;

cudaError_t set_hold_scan(int hold) { return cudaMemcpyToSymbol(g_hold_scan, &hold, sizeof(int)); }

// Rounds of the bounded wait for the scanning CTA (each about 0.1-0.2 us of
// sleep: about a second in all), after which the waiting CTA raises
// ERR_TIMEOUT and returns.
constexpr int SCAN_WAIT = 1 << 23;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// precise render record (see record_item_quad), written in double-float
//
// The ray-splat solve u ~ adj(T') (x - xc, y - yc, 1) is evaluated per pixel
// in binary32, but the adjugate itself is computed here in double-float from
// the binary32 inputs and rounded once: for a surfel seen nearly edge-on the
// intersection amplifies a relative error e in T by about (depth / size) /
// cos(view angle), so a binary32 chain (the binning mirror above) would put
// ~1e-3 relative error into alpha.  The binning record keeps the binary32
// values; only the render record r0..r2 and the rescale r3.w change.
// With n2 = |q|^2, R(q/|q|) = R'(q) / n2 where R' is the homogeneous
// (unnormalised) rotation polynomial, so n2 * T = K [r_u Rv t_u', r_v Rv t_v',
// n2 (Rv p + t)] needs no square root; its adjugate is n2^2 adj(T).
// ---------------------------------------------------------------------------
__device__ __forceinline__ df shfl_df(df v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src, 4), __shfl_sync(0xffffffffu, v.lo, src, 4)};
}

// One quad of lanes per item (j = lane & 3): lane j < 3 forms column j of the
// shifted n2 T' (the two tangent columns and the centre column), the quad
// exchanges the columns, and lane r < 3 forms adjugate row r; the operations
// and their order are those of a single-thread evaluation, so the record
// does not depend on the split.  Every lane of the warp must call this
// (shuffles); `valid` false computes nothing that is stored.
__device__ void record_item_quad(const Cams& cams, const RParams& P, const float* __restrict__ means,
                                 const float* __restrict__ scales, const float* __restrict__ quats,
                                 float4* __restrict__ rec, uint32_t item, bool valid) {
    const int j = threadIdx.x & 3, q0 = (threadIdx.x & 31) & ~3;
    const int view = view_of_item(item, P.N);
    const int64_t s = (int64_t)item - (int64_t)view * P.N;
    const CamDev& cam = cams.c[view];
    float4* rr = rec + 4 * (size_t)item;
    const float xc = rr[0].w, yc = rr[1].w;
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(quats) + s);
    const float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
    const df ww = two_prod(qw, qw), xx = two_prod(qx, qx), yy = two_prod(qy, qy), zz = two_prod(qz, qz);
    const df n2 = dadd(dadd(ww, xx), dadd(yy, zz));
    // column j of n2 T (camera frame, before the intrinsics): R t_u' r_u,
    // R t_v' r_v or n2 (R p + t); straight-line code with selects, so the
    // quad's lanes do not diverge
    const df xy = two_prod(qx, qy), wz = two_prod(qw, qz), xz = two_prod(qx, qz), wy = two_prod(qw, qy);
    const df yz = two_prod(qy, qz), wx = two_prod(qw, qx);
    const df tu[3] = {dsub(dadd(ww, xx), dadd(yy, zz)), dmulf(dadd(xy, wz), 2.0f), dmulf(dsub(xz, wy), 2.0f)};
    const df tv[3] = {dmulf(dsub(xy, wz), 2.0f), dsub(dadd(ww, yy), dadd(xx, zz)), dmulf(dadd(yz, wx), 2.0f)};
    const df pm[3] = {dfrom(means[3 * s]), dfrom(means[3 * s + 1]), dfrom(means[3 * s + 2])};
    df v[3], e[3], col[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = j == 0 ? tu[i] : (j == 1 ? tv[i] : pm[i]);
    dmvec(cam.R, v, e);
    const float sj = scales[2 * s + (j == 1 ? 1 : 0)];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const df a = dmulf(e[i], sj), b = dmul(dadd(e[i], dfrom(cam.t[i])), n2);
        col[i] = j < 2 ? a : b;
    }
    // column j of n2 T, shifted about (xc, yc)
    df dj[3];
    {
        const df cx = dadd(dmulf(col[0], cam.fx), dmulf(col[2], cam.cx));
        const df cy = dadd(dmulf(col[1], cam.fy), dmulf(col[2], cam.cy));
        dj[0] = dsub(cx, dmulf(col[2], xc));
        dj[1] = dsub(cy, dmulf(col[2], yc));
        dj[2] = col[2];
    }
    df d[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 3; ++i) d[c][i] = shfl_df(dj[i], q0 + c);
    // adjugate row j: m_j = d_{j+1} x d_{j+2} (operands picked by selects: a
    // dynamic index would put d in local memory)
    const int r = j < 3 ? j : 0;
    df da[3], db[3], m[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        da[i] = r == 0 ? d[1][i] : (r == 1 ? d[2][i] : d[0][i]);
        db[i] = r == 0 ? d[2][i] : (r == 1 ? d[0][i] : d[1][i]);
    }
    dcross(da, db, m);
    float mx = j < 3 ? fmaxf(fmaxf(fabsf(m[0].hi), fabsf(m[1].hi)), fabsf(m[2].hi)) : 0.0f;
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1, 4));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2, 4));
    // lane 0: det(n2 T') from row 0
    const df det = dadd(dadd(dmul(d[0][0], m[0]), dmul(d[0][1], m[1])), dmul(d[0][2], m[2]));
    int ex = 0;
    if (mx > 0.0f) frexp32(mx, &ex);
    // hit depth det(T') / c2: with M = 2^-ex n2^2 adj(T'), store 2^-ex det(n2 T') / n2
    const float detr = __shfl_sync(0xffffffffu, ldexp32(fdv(det.hi, n2.hi), -ex), q0);
    if (!valid || !(mx > 0.0f)) return;  // after the last shuffle: every lane took part
    if (j < 3)
        rr[j] = make_float4(ldexp32(m[0].hi, -ex), ldexp32(m[1].hi, -ex), ldexp32(m[2].hi, -ex),
                            j == 0 ? xc : (j == 1 ? yc : detr));
    // total scale of M relative to adj(T' of the normalised surfel)
    if (j == 0) rr[3].w = ldexp32(fm(n2.hi, n2.hi), -ex);
}

constexpr int EMIT_BATCH = 8;

// one slot in each of tiles tb[0, n) for `item`: all cursor atomics first, then the stores
__device__ __forceinline__ void emit_batch(uint32_t* __restrict__ cursor, uint32_t* __restrict__ list,
                                           const uint32_t* tb, int n, uint32_t item, int64_t cap, int ntiles,
                                           Status* st) {
    uint32_t pos[EMIT_BATCH];
#pragma unroll
    for (int j = 0; j < EMIT_BATCH; ++j)
        if (j < n) pos[j] = in_bounds(st, SITE_TILE, tb[j], ntiles) ? atomicAdd(&cursor[(size_t)tb[j] * TC_STRIDE], 1u) : ~0u;
#pragma unroll
    for (int j = 0; j < EMIT_BATCH; ++j)
        if (j < n && pos[j] < (uint32_t)cap) list[pos[j]] = item;
}

// ---------------------------------------------------------------------------
// k_emit: writes every bounded visible item into one slot of each of its
// tiles (slot order is arbitrary; the per-tile sort restores a total order)
// and replaces the render records by their double-float versions.
//   scan:         the first CTA to take the ticket scans the per-tile counts
//                 into ranges and emit cursors and publishes them (release
//                 store of a flag); it never waits, so the others' bounded
//                 wait for the flag ends however the CTAs are scheduled;
//   records:      one quad of lanes per narrow, wide or unbounded item (they
//                 need no ranges, so they run while the scan does);
//   narrow items: 32 per warp, their (item, outer line) units spread over
//                 the lanes; each lane emits its line's tiles;
//   wide items:   one warp per (item, outer line), lanes over the line's tiles;
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_emit(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                                              const BinRec* __restrict__ binrec, const uint32_t* __restrict__ vis_list,
                                              const uint32_t* __restrict__ wide_list,
                                              const uint32_t* __restrict__ unb_list, uint32_t* __restrict__ cursor,
                                              int2* __restrict__ ranges, int32_t* __restrict__ order,
                                              uint32_t* __restrict__ list, const float* __restrict__ means,
                                              const float* __restrict__ scales, const float* __restrict__ quats,
                                              float4* __restrict__ rec, Status* __restrict__ st, int max_lines) {
    __shared__ BinRec s_br[256];
    __shared__ uint32_t s_item[256];
    __shared__ int s_pre[256];
    __shared__ int s_scanner, s_go;
    if (st->err) return;
    Status* const stw = st;
    if (threadIdx.x == 0) s_scanner = atomicAdd(&st->scan_ticket, 1u) == 0u;
    __syncthreads();
    if (s_scanner) {
        scan_tiles(cams, P, cursor, ranges, st);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0 && !g_hold_scan) st_release(&st->scan_done, 1u);
        heavy_first_order(cams, ranges, order);
    }
    const int lane = threadIdx.x & 31;
    const int wb = threadIdx.x & ~31;
    const WarpLines wl{s_br + wb, s_item + wb, s_pre + wb};
    const uint32_t nvis = st->nvis, nwide = st->nwide;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    uint32_t nunb = 0;
    for (int v = 0; v < cams.n; ++v) nunb += st->unb_cnt[v];
    // render records of all visible items (narrow, wide, unbounded), one quad
    // of lanes each, from the lowest threads up (warp-uniform loop)
    const uint32_t nrec = nvis + nwide + nunb;
    for (int64_t base = (gtid >> 5) * 8; base < nrec; base += (gstride >> 5) * 8) {
        const int64_t ri = base + (lane >> 2);
        const bool valid = ri < nrec;
        uint32_t item = 0;
        bool ok = valid && in_bounds(stw, SITE_VIS_LIST, ri, P.n_items);
        if (ok) {
            if (ri < nvis) {
                item = vis_list[ri];
            } else if (ri < (int64_t)nvis + nwide) {
                item = wide_list[ri - nvis];
            } else {
                uint32_t k = (uint32_t)(ri - nvis - nwide);
                int v = 0;
                while (FSS_CHECKED(v < cams.n) && k >= st->unb_cnt[v]) k -= st->unb_cnt[v++];
                ok = in_bounds(stw, SITE_VIS_LIST, v, cams.n) && in_bounds(stw, SITE_VIS_LIST, k, P.N);
                item = ok ? unb_list[(int64_t)v * P.N + k] : 0u;
            }
            ok = ok && in_bounds(stw, SITE_ITEM, item, P.n_items);
        }
        record_item_quad(cams, P, means, scales, quats, rec, ok ? item : 0u, valid && ok);
    }
    // the emit cursors: published by the scanning CTA (bounded wait)
    if (threadIdx.x == 0) {
        bool done = s_scanner != 0;
        for (int i = 0; !done && i < SCAN_WAIT; ++i) {
            done = ld_acquire(&st->scan_done) != 0u;
            if (!done) __nanosleep(128);
        }
        if (!done) atomicOr(&st->err, ERR_TIMEOUT);
        s_go = done && !(ld_acquire(reinterpret_cast<const uint32_t*>(&st->err)) & ERR_CAPACITY);
    }
    __syncthreads();
    if (!s_go) return;
    // narrow items, 32 per warp from the highest warps down (so that they run
    // beside the records); each lane emits one line's tiles in batches of
    // EMIT_BATCH, whose cursor atomics are in flight together
    const int64_t warps = gstride >> 5;
    for (int64_t c0 = (warps - 1 - (gtid >> 5)) * 32; c0 < nvis; c0 += warps * 32) {  // warp-uniform
        const int64_t i = c0 + lane;
        bool ok = i < nvis && in_bounds(stw, SITE_VIS_LIST, i, P.n_items);
        const uint32_t item = ok ? vis_list[i] : 0u;
        ok = ok && in_bounds(stw, SITE_ITEM, item, P.n_items);
        int nl = 0;
        if (ok) {
            const BinRec r = binrec[item];
            wl.br[lane] = r;
            nl = lines_of(r, P.bin_mode).n;
        }
        wl.item[lane] = item;
        const int total = warp_line_prefix(wl, nl);
        warp_lines(cams, P, wl, total, [&](int, uint32_t it, const CamDev& cam, bool rows, int o, int a, int b) {
            uint32_t tb[EMIT_BATCH];
            int nb = 0;
            for (int k = a; k <= b; ++k) {
                const int tx = rows ? k : o, ty = rows ? o : k;
                tb[nb++] = (uint32_t)(cam.tile_off + ty * cam.tiles_x + tx);
                if (nb == EMIT_BATCH) {
                    emit_batch(cursor, list, tb, nb, it, P.pair_cap, cams.total_tiles, stw);
                    nb = 0;
                }
            }
            emit_batch(cursor, list, tb, nb, it, P.pair_cap, cams.total_tiles, stw);
        });
        __syncwarp();  // the slices are reused by the warp's next chunk
    }
    // wide items: one warp per (item, outer line), lanes over the line's tiles,
    // so that a surfel spanning many tiles is spread over many warps
    const int64_t units = (int64_t)nwide * max_lines;
    for (int64_t u = gtid >> 5; u < units; u += warps) {
        const int64_t wi = u / max_lines;
        const int li = (int)(u - wi * max_lines);
        if (!in_bounds(stw, SITE_VIS_LIST, wi, P.n_items)) break;
        const uint32_t item = wide_list[wi];
        if (!in_bounds(stw, SITE_ITEM, item, P.n_items)) continue;
        const BinRec r = binrec[item];
        const Lines L = lines_of(r, P.bin_mode);
        if (li >= L.n) continue;  // warp-uniform
        const CamDev& cam = cams.c[view_of_item(item, P.N)];
        const int o = L.first + li;
        int a, b;
        if (!line_interval(r, L, P.ts, o, a, b)) continue;
        for (int k = a + lane; k <= b; k += 32) {
            const int tx = L.rows ? k : o, ty = L.rows ? o : k;
            const int tt = cam.tile_off + ty * cam.tiles_x + tx;
            if (!in_bounds(stw, SITE_TILE, tt, cams.total_tiles)) continue;
            const uint32_t pos = atomicAdd(&cursor[(size_t)tt * TC_STRIDE], 1u);
            if (pos < (uint32_t)P.pair_cap) list[pos] = item;
        }
    }
}

}  // namespace fss
