// C ABI of the rasterizer library (include/fss.h): argument validation,
// workspace layout and kernel launches.  No entry point allocates memory.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "fss_internal.cuh"
#include "kernels.cuh"

namespace fss {
namespace {

thread_local std::string g_err;

fss_status fail(fss_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
fss_status fail(fss_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

fss_status cuda_fail(cudaError_t e, const char* where) {
    return fail(FSS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int num_sms_current() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
    return n;
}

fss_status check_params(const fss_params* p) {
    if (!p) return fail(FSS_ERR_INVALID_ARG, "params is NULL");
    if (p->tile_size != 8 && p->tile_size != 16 && p->tile_size != 32)
        return fail(FSS_ERR_UNSUPPORTED, "tile_size %d not in {8,16,32}", p->tile_size);
    if (p->K < 0 || p->K > FSS_MAX_K) return fail(FSS_ERR_UNSUPPORTED, "K %d not in [0,%d]", p->K, FSS_MAX_K);
    if (p->bin_mode < FSS_BIN_AABB || p->bin_mode > FSS_BIN_ACCU)
        return fail(FSS_ERR_INVALID_ARG, "bin_mode %d", p->bin_mode);
    if (p->stop_rule != FSS_STOP_TMIN && p->stop_rule != FSS_STOP_EXACT_TOPK)
        return fail(FSS_ERR_INVALID_ARG, "stop_rule %d", p->stop_rule);
    if ((p->feat_dtype != FSS_F32 && p->feat_dtype != FSS_BF16) || (p->out_dtype != FSS_F32 && p->out_dtype != FSS_BF16))
        return fail(FSS_ERR_INVALID_ARG, "feat_dtype/out_dtype must be FSS_F32 or FSS_BF16");
    const int vec = (p->feat_dtype == FSS_BF16 || p->out_dtype == FSS_BF16) ? 8 : 4;
    if (p->C < 4 || p->C > 512 || p->C % vec)
        return fail(FSS_ERR_UNSUPPORTED, "C %d must be a multiple of %d in [4,512]", p->C, vec);
    if (p->K == 0 && p->C > 128) return fail(FSS_ERR_UNSUPPORTED, "full accumulation (K=0) supports C <= 128");
    if (!(p->alpha_min > 0.0f) || !(p->alpha_max > p->alpha_min) || !(p->alpha_max < 1.0f))
        return fail(FSS_ERR_INVALID_ARG, "need 0 < alpha_min < alpha_max < 1");
    if (!(p->T_min >= 0.0f) || !(p->T_min < 1.0f)) return fail(FSS_ERR_INVALID_ARG, "need 0 <= T_min < 1");
    if (p->schedule != FSS_SCHED_GRID && p->schedule != FSS_SCHED_PERSISTENT)
        return fail(FSS_ERR_INVALID_ARG, "schedule %d", p->schedule);
    if (p->select != FSS_SELECT_TOPW && p->select != FSS_SELECT_FRONT)
        return fail(FSS_ERR_INVALID_ARG, "select %d", p->select);
    if (p->renorm != 0 && p->renorm != 1) return fail(FSS_ERR_INVALID_ARG, "renorm %d", p->renorm);
    if (p->renorm && p->K == 0) return fail(FSS_ERR_INVALID_ARG, "renorm needs K > 0");
    if (p->lowpass != 0 && p->lowpass != 1) return fail(FSS_ERR_INVALID_ARG, "lowpass %d", p->lowpass);
    if (p->color_mode != FSS_COLOR_RGB && p->color_mode != FSS_COLOR_SH)
        return fail(FSS_ERR_INVALID_ARG, "color_mode %d", p->color_mode);
    if (p->color_mode == FSS_COLOR_SH && (p->sh_degree < 0 || p->sh_degree > 3))
        return fail(FSS_ERR_UNSUPPORTED, "sh_degree %d not in [0,3]", p->sh_degree);
    return FSS_OK;
}

fss_status make_cams(const fss_camera* cams, int32_t n, int ts, Cams& out) {
    if (!cams) return fail(FSS_ERR_INVALID_ARG, "cams is NULL");
    if (n < 1 || n > FSS_MAX_CAMS) return fail(FSS_ERR_UNSUPPORTED, "n_cams %d not in [1,%d]", n, FSS_MAX_CAMS);
    std::memset(&out, 0, sizeof out);
    out.n = n;
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < n; ++v) {
        const fss_camera& c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
            return fail(FSS_ERR_UNSUPPORTED, "camera %d: size %dx%d not in [1,16384]^2", v, c.width, c.height);
        if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !(c.near_plane > 0.0f))
            return fail(FSS_ERR_INVALID_ARG, "camera %d: need fx, fy, near_plane > 0", v);
        CamDev& d = out.c[v];
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) d.R[3 * r + k] = c.viewmat[4 * r + k];
            d.t[r] = c.viewmat[4 * r + 3];
        }
        d.near_plane = c.near_plane;
        d.W = c.width; d.H = c.height;
        d.tiles_x = (c.width + ts - 1) / ts;
        d.tiles_y = (c.height + ts - 1) / ts;
        d.tile_off = (int32_t)tiles;
        d.pix_off = pix;
        tiles += (int64_t)d.tiles_x * d.tiles_y;
        pix += (int64_t)c.width * c.height;
    }
    if (tiles > (1 << 30)) return fail(FSS_ERR_UNSUPPORTED, "too many tiles");
    out.total_tiles = (int32_t)tiles;
    out.total_pix = pix;
    return FSS_OK;
}

RParams make_rparams(const fss_params* p, const Cams& cams, int64_t N, int64_t cap) {
    RParams r;
    r.ts = p->tile_size; r.K = p->K; r.bin_mode = p->bin_mode; r.stop_rule = p->stop_rule;
    r.alpha_min = p->alpha_min; r.alpha_max = p->alpha_max; r.T_min = p->T_min;
    r.feat_dtype = p->feat_dtype; r.out_dtype = p->out_dtype; r.C = p->C;
    r.select = p->select;
    r.renorm = p->renorm;
    r.lowpass = p->lowpass;
    r.color_sh = p->color_mode == FSS_COLOR_SH;
    r.sh_deg = r.color_sh ? p->sh_degree : 0;
    for (int k = 0; k < 3; ++k) r.bg[k] = p->bg_rgb[k];
    r.N = N;
    r.n_items = N * cams.n;
    r.pair_cap = cap;
    return r;
}

Layout make_layout(const RParams& P, const Cams& cams) {
    Layout L;
    size_t sz[REG_COUNT_ALL] = {};
    const size_t ni = (size_t)P.n_items, N = (size_t)P.N, cap = (size_t)P.pair_cap;
    sz[REG_STATUS] = sizeof(Status);
    sz[REG_REC] = ni * 64;
    sz[REG_BINREC] = ni * sizeof(BinRec);
    sz[REG_COUNT] = ni * 4;
    sz[REG_RANGES] = (size_t)cams.total_tiles * 8;
    sz[REG_LIST] = cap * 4;
    sz[REG_COUNTERS] = 0;  // inside the status block
    sz[REG_TILECNT] = (size_t)cams.total_tiles * 4 * TC_STRIDE;
    sz[REG_SORTTMP] = cap * 16;
    sz[REG_GRAD_ITEM] = (size_t)cams.n * N * GRAD_STRIDE * 4;
    sz[REG_FEAT_ACC] = N * (size_t)P.C * 4;
    sz[REG_DOTS] = (size_t)cams.total_pix * (size_t)P.K * 4;
    sz[REG_VIS] = ni * 4;
    sz[REG_UNB] = ni * 4;
    sz[REG_SLOT] = N * 4;
    sz[REG_WIDE] = ni * 4;
    sz[REG_MASK] = cap * 4;
    sz[REG_SLOT_SURF] = N * 4;
    sz[REG_DIR] = P.color_sh ? ni * 16 : 0;
    sz[REG_COLOR] = P.color_sh ? ni * 12 : 0;
    sz[REG_ORDER] = (size_t)cams.total_tiles * 4;
    size_t off = 0;
    for (int r = 0; r < REG_COUNT_ALL; ++r) {
        L.off[r] = off;
        L.size[r] = sz[r];
        off += align256(sz[r]) + GUARD_BYTES;  // check build: the region's canary follows it
    }
    L.off[REG_COUNTERS] = L.off[REG_STATUS] + STATUS_CLEAR_OFF;
    L.size[REG_COUNTERS] = sizeof(((Status*)0)->counters);
    L.total = off;
    return L;
}

struct Ctx {
    Cams cams;
    RParams P;
    Layout L;
    unsigned char* ws;
    template <typename T>
    T* at(int r) const { return reinterpret_cast<T*>(ws + L.off[r]); }
};

fss_status prepare(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N, int64_t cap,
                   void* workspace, Ctx& ctx) {
    fss_status s = check_params(params);
    if (s != FSS_OK) return s;
    if ((s = make_cams(cams, n_cams, params->tile_size, ctx.cams)) != FSS_OK) return s;
    if (N < 0 || N > ((int64_t)1 << 30)) return fail(FSS_ERR_UNSUPPORTED, "N %lld not in [0, 2^30]", (long long)N);
    if (N * n_cams >= ((int64_t)1 << 32)) return fail(FSS_ERR_UNSUPPORTED, "N * n_cams must be < 2^32");
    if (cap < 0 || cap >= ((int64_t)1 << 31)) return fail(FSS_ERR_UNSUPPORTED, "pair_capacity not in [0, 2^31)");
    ctx.P = make_rparams(params, ctx.cams, N, cap);
    ctx.L = make_layout(ctx.P, ctx.cams);
    ctx.ws = reinterpret_cast<unsigned char*>(workspace);
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255))
        return fail(FSS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    ctx.cams.tile_order = workspace ? ctx.at<int32_t>(REG_ORDER) : nullptr;
    return FSS_OK;
}

bool misaligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15); }

const char* const kRegionNames[REG_COUNT_ALL] = {
    "status", "records", "binning records", "tile counts per item", "tile ranges", "pair list", "counters",
    "tile cursors", "sort scratch", "gradient rows", "feature-gradient rows", "dots", "visible items",
    "unbounded items", "gradient slots", "wide items", "warp masks", "slot surfels", "directions", "item colours",
    "tile order"};
const char* const kSiteNames[SITE_COUNT] = {"none", "tile id", "visible-item list slot", "gradient slot",
                                            "tile range", "pair-list item", "sort scratch",
                                            "saved list position", "feature row"};

// check build: canary of region r (GUARD_BYTES after its aligned end)
size_t guard_off(const Layout& L, int r) { return L.off[r] + align256(L.size[r]); }

// check build: writes every region's canary and marks the status block
cudaError_t arm_guards(const Ctx& ctx, cudaStream_t st) {
    if (!GUARD_BYTES) return cudaSuccess;
    for (int r = 0; r < REG_COUNT_ALL; ++r) {
        if (r == REG_COUNTERS) continue;  // inside the status block
        cudaError_t e = cudaMemsetAsync(ctx.ws + guard_off(ctx.L, r), GUARD_BYTE, GUARD_BYTES, st);
        if (e != cudaSuccess) return e;
    }
    return cudaMemsetAsync(ctx.ws + ctx.L.off[REG_STATUS] + offsetof(Status, guards), GUARD_BYTE, sizeof(uint32_t), st);
}

// check build: the first region whose canary was overwritten, or -1 (after a synchronising read)
int broken_guard(const Ctx& ctx, cudaStream_t st, cudaError_t& e) {
    e = cudaSuccess;
    if (!GUARD_BYTES) return -1;
    unsigned char buf[REG_COUNT_ALL][GUARD_BYTES ? GUARD_BYTES : 1];
    for (int r = 0; r < REG_COUNT_ALL && e == cudaSuccess; ++r)
        if (r != REG_COUNTERS)
            e = cudaMemcpyAsync(buf[r], ctx.ws + guard_off(ctx.L, r), GUARD_BYTES, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return -1;
    for (int r = 0; r < REG_COUNT_ALL; ++r) {
        if (r == REG_COUNTERS) continue;
        for (size_t k = 0; k < GUARD_BYTES; ++k)
            if (buf[r][k] != GUARD_BYTE) return r;
    }
    return -1;
}

}  // namespace

// Records `msg` as the calling thread's last error (for units outside this file).
fss_status set_error(fss_status s, const char* msg) { return fail(s, "%s", msg); }

namespace {
thread_local cudaEvent_t* g_mark_ev = nullptr;
thread_local int g_mark_n = 0, g_mark_k = 0;
}  // namespace

bool kernel_marks_armed() { return g_mark_k < g_mark_n; }

namespace {
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int SIDE_DEVS = 64;
// Per thread and device, created at the thread's first eager backward call on
// the device and released when the thread exits (errors ignored: when the
// process exits, the runtime may already be shutting down).
struct SideStreams {
    SideStream d[SIDE_DEVS];
    ~SideStreams() {
        for (SideStream& x : d) {
            if (x.s) (void)cudaStreamDestroy(x.s);
            if (x.fork) (void)cudaEventDestroy(x.fork);
            if (x.join) (void)cudaEventDestroy(x.join);
        }
        (void)cudaGetLastError();
    }
};
thread_local SideStreams g_side;
}  // namespace

bool side_stream(cudaStream_t s, cudaStream_t& side, cudaEvent_t& fork, cudaEvent_t& join) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SIDE_DEVS) {
        (void)cudaGetLastError();
        return false;
    }
    SideStream& x = g_side.d[dev];
    if (x.s == nullptr) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            (void)cudaGetLastError();
            return false;
        }
        cudaStream_t ns = nullptr;
        cudaEvent_t ef = nullptr, ej = nullptr;
        if (cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ef, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ej, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            if (ns) (void)cudaStreamDestroy(ns);
            if (ef) (void)cudaEventDestroy(ef);
            return false;
        }
        x.s = ns;
        x.fork = ef;
        x.join = ej;
    }
    side = x.s;
    fork = x.fork;
    join = x.join;
    return true;
}

void kernel_mark(cudaStream_t s) {
    if (g_mark_k >= g_mark_n) return;
    // an external record becomes a node of a graph being captured; outside a
    // capture the plain record is the valid form
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e == cudaSuccess)
        e = cs == cudaStreamCaptureStatusActive
                ? cudaEventRecordWithFlags(g_mark_ev[g_mark_k], s, cudaEventRecordExternal)
                : cudaEventRecord(g_mark_ev[g_mark_k], s);
    ++g_mark_k;
    if (e != cudaSuccess) {  // timing must never fail a compute call: drop the hook
        (void)cudaGetLastError();
        g_mark_n = g_mark_k = 0;
        g_mark_ev = nullptr;
    }
}

}  // namespace fss

using namespace fss;

extern "C" {

fss_status fss_default_params(fss_params* p) {
    if (!p) return fail(FSS_ERR_INVALID_ARG, "params is NULL");
    std::memset(p, 0, sizeof *p);
    p->tile_size = 16;
    p->K = 8;
    p->bin_mode = FSS_BIN_ACCU;
    p->stop_rule = FSS_STOP_TMIN;
    p->alpha_min = 1.0f / 255.0f;
    p->alpha_max = 0.99f;
    p->T_min = 1e-4f;
    p->feat_dtype = FSS_F32;
    p->out_dtype = FSS_F32;
    p->C = 16;
    return FSS_OK;
}

fss_status fss_workspace_size(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                              int64_t pair_capacity, size_t* bytes) {
    Ctx ctx;
    fss_status s = prepare(params, cams, n_cams, N, pair_capacity, nullptr, ctx);
    if (s != FSS_OK) return s;
    if (!bytes) return fail(FSS_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = ctx.L.total;
    return FSS_OK;
}

fss_status fss_saved_size(const fss_params* params, const fss_camera* cams, int32_t n_cams, size_t* bytes) {
    fss_status s = check_params(params);
    if (s != FSS_OK) return s;
    Cams c;
    if ((s = make_cams(cams, n_cams, params->tile_size, c)) != FSS_OK) return s;
    if (!bytes) return fail(FSS_ERR_INVALID_ARG, "bytes is NULL");
    const size_t px = (size_t)c.total_pix;
    *bytes = align256(px * params->K * 4) * 2 + align256(px * 4);
    return FSS_OK;
}

fss_status fss_workspace_region(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                                int64_t pair_capacity, int32_t which, size_t* offset, size_t* bytes) {
    Ctx ctx;
    fss_status s = prepare(params, cams, n_cams, N, pair_capacity, nullptr, ctx);
    if (s != FSS_OK) return s;
    if (which < 0 || which >= REG_COUNT_ALL) return fail(FSS_ERR_INVALID_ARG, "region %d", which);
    if (offset) *offset = ctx.L.off[which];
    if (bytes) *bytes = ctx.L.size[which];
    return FSS_OK;
}

fss_status fss_project_bin(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                           const float* means, const float* scales, const float* quats, const float* opac,
                           void* workspace, int64_t pair_capacity, fss_stream_t stream) {
    Ctx ctx;
    fss_status s = prepare(params, cams, n_cams, N, pair_capacity, workspace, ctx);
    if (s != FSS_OK) return s;
    if (!workspace) return fail(FSS_ERR_INVALID_ARG, "workspace is NULL");
    if (N > 0 && (!means || !scales || !quats || !opac)) return fail(FSS_ERR_INVALID_ARG, "NULL surfel input");
    if ((reinterpret_cast<uintptr_t>(quats) & 15) || (reinterpret_cast<uintptr_t>(scales) & 7))
        return fail(FSS_ERR_INVALID_ARG, "quats must be 16-byte and scales 8-byte aligned");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    // clear the per-frame part of the status block and the gradient slots
    e = cudaMemsetAsync(ctx.ws + ctx.L.off[REG_STATUS] + STATUS_CLEAR_OFF, 0, sizeof(Status) - STATUS_CLEAR_OFF, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset status");
    if (N > 0) {
        e = cudaMemsetAsync(ctx.ws + ctx.L.off[REG_SLOT], 0xff, (size_t)N * 4, st);
        if (e != cudaSuccess) return cuda_fail(e, "memset slots");
    }
    e = cudaMemsetAsync(ctx.ws + ctx.L.off[REG_TILECNT], 0, (size_t)ctx.cams.total_tiles * 4 * TC_STRIDE, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset tile counts");
    if ((e = arm_guards(ctx, st)) != cudaSuccess) return cuda_fail(e, "memset canaries");
    const int sms = num_sms_current();
    Status* stp = ctx.at<Status>(REG_STATUS);
    const int64_t items = ctx.P.n_items;
    const int64_t blocks = std::max<int64_t>(1, (items + 1023) / 1024);  // PROJ_ITEMS items per CTA
    k_project<<<(unsigned)blocks, 256, 0, st>>>(ctx.cams, ctx.P, means, scales, quats, opac, ctx.at<float4>(REG_REC),
                                               ctx.at<BinRec>(REG_BINREC), ctx.at<uint32_t>(REG_COUNT),
                                               ctx.at<uint32_t>(REG_TILECNT), ctx.at<uint32_t>(REG_VIS),
                                               ctx.at<uint32_t>(REG_WIDE), ctx.at<uint32_t>(REG_UNB),
                                               ctx.at<int32_t>(REG_SLOT), ctx.at<int32_t>(REG_SLOT_SURF), stp);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_project");
    kernel_mark(st);
    // one resident wave: records run from the lowest threads up, tile emission
    // from the highest down, so both start at once; one CTA scans the tile
    // counts first
    int emit_per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&emit_per_sm, k_emit, 256, 0)) != cudaSuccess)
        return cuda_fail(e, "occupancy k_emit");
    const unsigned emit_blocks = (unsigned)(std::max(1, emit_per_sm) * sms);
    int max_lines = 1;  // most outer tile lines (rows or columns) of any view
    for (int v = 0; v < ctx.cams.n; ++v)
        max_lines = std::max(max_lines, std::max(ctx.cams.c[v].tiles_x, ctx.cams.c[v].tiles_y));
    k_emit<<<emit_blocks, 256, 0, st>>>(ctx.cams, ctx.P, ctx.at<BinRec>(REG_BINREC), ctx.at<uint32_t>(REG_VIS),
                                    ctx.at<uint32_t>(REG_WIDE), ctx.at<uint32_t>(REG_UNB),
                                    ctx.at<uint32_t>(REG_TILECNT), ctx.at<int2>(REG_RANGES),
                                    ctx.at<int32_t>(REG_ORDER), ctx.at<uint32_t>(REG_LIST), means, scales, quats,
                                    ctx.at<float4>(REG_REC), stp, max_lines);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_emit");
    kernel_mark(st);
    if (ctx.P.color_sh) {
        e = launch_sh_dir(ctx.cams, ctx.P, ctx.at<uint32_t>(REG_VIS), ctx.at<uint32_t>(REG_WIDE),
                          ctx.at<uint32_t>(REG_UNB), means, ctx.at<float4>(REG_DIR), stp, sms, st);
        if (e != cudaSuccess) return cuda_fail(e, "k_sh_dir");
    }
    return FSS_OK;
}

namespace {

fss_status launch_sort(Ctx& ctx, cudaStream_t st) {
    k_tile_sort<<<ctx.cams.total_tiles, SORT_THREADS, 0, st>>>(ctx.cams, ctx.P, ctx.at<float4>(REG_REC),
                                                      ctx.at<BinRec>(REG_BINREC), ctx.at<int2>(REG_RANGES),
                                                      ctx.at<uint32_t>(REG_LIST), ctx.at<uint32_t>(REG_UNB),
                                                      ctx.at<uint64_t>(REG_SORTTMP), ctx.at<uint32_t>(REG_MASK),
                                                      ctx.at<Status>(REG_STATUS));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_tile_sort");
    kernel_mark(st);
    return FSS_OK;
}

}  // namespace

fss_status fss_sort(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N, void* workspace,
                    int64_t pair_capacity, fss_stream_t stream) {
    Ctx ctx;
    fss_status s = prepare(params, cams, n_cams, N, pair_capacity, workspace, ctx);
    if (s != FSS_OK) return s;
    if (!workspace) return fail(FSS_ERR_INVALID_ARG, "workspace is NULL");
    return launch_sort(ctx, reinterpret_cast<cudaStream_t>(stream));
}

fss_status fss_render_forward(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                              void* workspace, int64_t pair_capacity, const float* rgb, const void* feats,
                              void* out_feat, float* out_rgb, float* out_T, int32_t* out_topk_id, void* saved,
                              fss_stream_t stream) {
    return fss_render_forward_aux(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb,
                                  out_T, out_topk_id, saved, nullptr, stream);
}

namespace {

// the training loss of fss_render_forward_loss
struct LossIn {
    const void* Ft;
    const float* rgbt;
    float wf, wc;
    void* dF;
    float* drgb;
    double* loss;
};

fss_status render_forward_impl(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                               void* workspace, int64_t pair_capacity, const float* rgb, const void* feats,
                               void* out_feat, float* out_rgb, float* out_T, int32_t* out_topk_id, void* saved,
                               const fss_aux_outputs* aux, const LossIn* li, bool sort, fss_stream_t stream) {
    Ctx ctx;
    fss_status s = prepare(params, cams, n_cams, N, pair_capacity, workspace, ctx);
    if (s != FSS_OK) return s;
    if (!workspace) return fail(FSS_ERR_INVALID_ARG, "workspace is NULL");
    if (N > 0 && !rgb) return fail(FSS_ERR_INVALID_ARG, "rgb is NULL");
    if (out_feat && N > 0 && !feats) return fail(FSS_ERR_INVALID_ARG, "feats is NULL while out_feat is given");
    if (misaligned16(feats) || misaligned16(out_feat))
        return fail(FSS_ERR_INVALID_ARG, "feats and out_feat must be 16-byte aligned");
    FwdArgs a;
    std::memset(&a, 0, sizeof a);
    a.rec = ctx.at<float4>(REG_REC);
    a.binrec = ctx.at<BinRec>(REG_BINREC);
    a.ranges = ctx.at<int2>(REG_RANGES);
    a.list = ctx.at<uint32_t>(REG_LIST);
    a.masks = ctx.at<uint32_t>(REG_MASK);
    a.rgb = params->color_mode == FSS_COLOR_SH ? ctx.at<float>(REG_COLOR) : rgb;
    a.feats = feats;
    a.out_feat = out_feat;
    a.out_rgb = out_rgb;
    a.out_T = out_T;
    a.out_ids = params->K > 0 ? out_topk_id : nullptr;
    if (saved) {
        const size_t px = (size_t)ctx.cams.total_pix;
        unsigned char* sv = reinterpret_cast<unsigned char*>(saved);
        a.saved_pos = params->K > 0 ? reinterpret_cast<int32_t*>(sv) : nullptr;
        a.saved_w = params->K > 0 ? reinterpret_cast<float*>(sv + align256(px * params->K * 4)) : nullptr;
        a.saved_nstop = reinterpret_cast<int32_t*>(sv + 2 * align256(px * params->K * 4));
    }
    AuxOut x{nullptr, nullptr, nullptr, nullptr};
    if (aux) x = AuxOut{aux->depth, aux->depth_median, aux->normal, aux->label};
    a.st = ctx.at<Status>(REG_STATUS);
    a.persistent = params->schedule == FSS_SCHED_PERSISTENT;
    if (a.persistent) {  // the queue head, so that a frame's forward may run more than once
        cudaError_t e = cudaMemsetAsync(ctx.ws + ctx.L.off[REG_STATUS] + offsetof(Status, work), 0, sizeof(uint32_t),
                                        reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(e, "memset work queue");
    }
    if (ctx.P.color_sh && N > 0) {  // this frame's item colours from the coefficients
        cudaError_t ec = launch_sh_color(ctx.cams, ctx.P, ctx.at<uint32_t>(REG_VIS), ctx.at<uint32_t>(REG_WIDE),
                                         ctx.at<uint32_t>(REG_UNB), ctx.at<float4>(REG_DIR), rgb,
                                         ctx.at<float>(REG_COLOR), a.st, num_sms_current(),
                                         reinterpret_cast<cudaStream_t>(stream));
        if (ec != cudaSuccess) return cuda_fail(ec, "k_sh_color");
    }
    const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n_pix = ctx.cams.total_pix;
    // the loss in the Top-K kernel's phase 2: the plain selection with K <= 8 and
    // the output in the feature type; otherwise the loss kernel after the render
    const bool fused = li && params->K > 0 && params->K <= 8 && params->select != FSS_SELECT_FRONT &&
                       !params->lowpass && !x.any() && params->out_dtype == params->feat_dtype;
    if (fused) {
        cudaError_t e = cudaMemsetAsync(li->loss, 0, sizeof(double), cs);
        if (e != cudaSuccess) return cuda_fail(e, "memset loss");
        if (n_pix > 0) {  // the scale factors exactly as the loss kernel forms them
            x.loss = LossOut{li->Ft, li->rgbt, li->dF, li->drgb, li->loss, 2.0f * li->wf / (float)(n_pix * params->C),
                             li->wf / (float)(n_pix * params->C), li->wc / (float)(n_pix * 3)};
            if (sort)  // each CTA sorts its tile first (the same regions as the sort kernel)
                x.sort = SortIn{ctx.at<BinRec>(REG_BINREC), ctx.at<uint32_t>(REG_LIST), ctx.at<uint32_t>(REG_MASK),
                                ctx.at<uint32_t>(REG_UNB), ctx.at<uint64_t>(REG_SORTTMP)};
        }
    }
    if (sort && !x.sort.list) {  // the sort kernel first
        const fss_status ss = launch_sort(ctx, cs);
        if (ss != FSS_OK) return ss;
    }
    cudaError_t e = launch_render_forward(ctx.cams, ctx.P, a, x, num_sms_current(), cs);
    if (e != cudaSuccess) return cuda_fail(e, "render_forward");
    if (li && !fused) {
        e = launch_loss(n_pix, params->C, params->out_dtype, out_feat, out_rgb, li->Ft, li->rgbt, li->wf, li->wc, li->dF,
                        li->drgb, li->loss, num_sms_current(), cs);
        if (e != cudaSuccess) return cuda_fail(e, "loss");
    }
    return FSS_OK;
}

}  // namespace

fss_status fss_render_forward_aux(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                                  void* workspace, int64_t pair_capacity, const float* rgb, const void* feats,
                                  void* out_feat, float* out_rgb, float* out_T, int32_t* out_topk_id, void* saved,
                                  const fss_aux_outputs* aux, fss_stream_t stream) {
    return render_forward_impl(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb, out_T,
                               out_topk_id, saved, aux, nullptr, false, stream);
}

fss_status fss_render_forward_loss(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                                   void* workspace, int64_t pair_capacity, const float* rgb, const void* feats,
                                   void* out_feat, float* out_rgb, float* out_T, int32_t* out_topk_id, void* saved,
                                   const void* feat_target, const float* rgb_target, float w_feat, float w_rgb,
                                   void* d_feat, float* d_rgb, double* loss, fss_stream_t stream) {
    if (!out_feat || !out_rgb || !feat_target || !rgb_target || !d_feat || !d_rgb || !loss)
        return fail(FSS_ERR_INVALID_ARG, "NULL loss argument (out_feat, out_rgb, targets, gradients, loss)");
    if (misaligned16(feat_target) || misaligned16(d_feat))
        return fail(FSS_ERR_INVALID_ARG, "feature buffers must be 16-byte aligned");
    const LossIn li{feat_target, rgb_target, w_feat, w_rgb, d_feat, d_rgb, loss};
    return render_forward_impl(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb, out_T,
                               out_topk_id, saved, nullptr, &li, false, stream);
}

fss_status fss_sort_render_forward_loss(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                                        void* workspace, int64_t pair_capacity, const float* rgb, const void* feats,
                                        void* out_feat, float* out_rgb, float* out_T, int32_t* out_topk_id,
                                        void* saved, const void* feat_target, const float* rgb_target, float w_feat,
                                        float w_rgb, void* d_feat, float* d_rgb, double* loss, fss_stream_t stream) {
    if (!out_feat || !out_rgb || !feat_target || !rgb_target || !d_feat || !d_rgb || !loss)
        return fail(FSS_ERR_INVALID_ARG, "NULL loss argument (out_feat, out_rgb, targets, gradients, loss)");
    if (misaligned16(feat_target) || misaligned16(d_feat))
        return fail(FSS_ERR_INVALID_ARG, "feature buffers must be 16-byte aligned");
    const LossIn li{feat_target, rgb_target, w_feat, w_rgb, d_feat, d_rgb, loss};
    return render_forward_impl(params, cams, n_cams, N, workspace, pair_capacity, rgb, feats, out_feat, out_rgb, out_T,
                               out_topk_id, saved, nullptr, &li, true, stream);
}

fss_status fss_render_backward(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                               void* workspace, int64_t pair_capacity, const float* means, const float* scales,
                               const float* quats, const float* opac, const float* rgb, const void* feats,
                               const void* saved, const float* out_T, const void* d_feat, const float* d_rgb,
                               const float* d_T, float* g_means, float* g_scales, float* g_quats, float* g_opac,
                               float* g_rgb, void* g_feat, fss_stream_t stream) {
    Ctx ctx;
    fss_status s = prepare(params, cams, n_cams, N, pair_capacity, workspace, ctx);
    if (s != FSS_OK) return s;
    if (!workspace || !saved || !out_T || !d_rgb) return fail(FSS_ERR_INVALID_ARG, "NULL workspace/saved/out_T/d_rgb");
    if (params->out_dtype != params->feat_dtype)
        return fail(FSS_ERR_UNSUPPORTED, "backward needs out_dtype == feat_dtype");
    if (params->K > 0 && params->C / (params->feat_dtype == FSS_BF16 ? 8 : 4) > 32)
        return fail(FSS_ERR_UNSUPPORTED, "Top-K backward supports C <= %d", params->feat_dtype == FSS_BF16 ? 256 : 128);
    if (N > 0 && (!means || !scales || !quats || !opac || !rgb || !feats || !d_feat))
        return fail(FSS_ERR_INVALID_ARG, "NULL surfel input or d_feat");
    if (misaligned16(feats) || misaligned16(d_feat) || misaligned16(g_feat))
        return fail(FSS_ERR_INVALID_ARG, "feats, d_feat and g_feat must be 16-byte aligned");
    BwdArgs a;
    std::memset(&a, 0, sizeof a);
    a.rec = ctx.at<float4>(REG_REC);
    a.binrec = ctx.at<BinRec>(REG_BINREC);
    a.ranges = ctx.at<int2>(REG_RANGES);
    a.list = ctx.at<uint32_t>(REG_LIST);
    a.masks = ctx.at<uint32_t>(REG_MASK);
    a.rgb = params->color_mode == FSS_COLOR_SH ? ctx.at<float>(REG_COLOR) : rgb;  // the forward's item colours
    a.feats = feats;
    const size_t px = (size_t)ctx.cams.total_pix;
    const unsigned char* sv = reinterpret_cast<const unsigned char*>(saved);
    a.saved_pos = params->K > 0 ? reinterpret_cast<const int32_t*>(sv) : nullptr;
    a.saved_w = params->K > 0 ? reinterpret_cast<const float*>(sv + align256(px * params->K * 4)) : nullptr;
    a.saved_nstop = reinterpret_cast<const int32_t*>(sv + 2 * align256(px * params->K * 4));
    a.out_T = out_T;
    a.d_feat = d_feat;
    a.d_rgb = d_rgb;
    a.d_T = d_T;
    a.dots = ctx.at<float>(REG_DOTS);
    a.grad_item = ctx.at<float>(REG_GRAD_ITEM);
    a.feat_acc = ctx.at<float>(REG_FEAT_ACC);
    a.splat_slot = ctx.at<int32_t>(REG_SLOT);
    a.slot_surf = ctx.at<int32_t>(REG_SLOT_SURF);
    a.means = means; a.scales = scales; a.quats = quats; a.opac = opac;
    a.g_means = g_means; a.g_scales = g_scales; a.g_quats = g_quats; a.g_opac = g_opac; a.g_rgb = g_rgb;
    a.g_feat = g_feat;
    a.st = ctx.at<Status>(REG_STATUS);
    a.persistent = params->schedule == FSS_SCHED_PERSISTENT;
    if (N == 0) return FSS_OK;
    cudaError_t e = launch_render_backward(ctx.cams, ctx.P, a, params->color_mode == FSS_COLOR_SH ? rgb : nullptr,
                                           num_sms_current(), reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "render_backward");
    return FSS_OK;
}

fss_status fss_read_status(const fss_params* params, const fss_camera* cams, int32_t n_cams, int64_t N,
                           void* workspace, int64_t pair_capacity, int64_t* num_pairs, fss_stream_t stream) {
    Ctx ctx;
    fss_status s = prepare(params, cams, n_cams, N, pair_capacity, workspace, ctx);
    if (s != FSS_OK) return s;
    if (!workspace) return fail(FSS_ERR_INVALID_ARG, "workspace is NULL");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Status h;
    cudaError_t e = cudaMemcpyAsync(&h, ctx.ws + ctx.L.off[REG_STATUS], sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "read status");
    if (num_pairs) *num_pairs = h.pairs_needed;
    if (GUARD_BYTES && h.guards == GUARD_WORD) {  // check build: the canaries of an armed workspace
        const int r = broken_guard(ctx, st, e);
        if (e != cudaSuccess) return cuda_fail(e, "read canaries");
        if (r >= 0) return fail(FSS_ERR_BOUNDS, "the canary after workspace region %d (%s) was overwritten", r,
                                kRegionNames[r]);
    }
    if (h.err) {
        e = cudaMemsetAsync(ctx.ws + ctx.L.off[REG_STATUS], 0, sizeof(int32_t), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "clear status");
        if (h.err & ERR_BOUNDS)
            return fail(FSS_ERR_BOUNDS, "device index check failed at %s: index %lld",
                        h.bounds_site < SITE_COUNT ? kSiteNames[h.bounds_site] : "?", (long long)h.bounds_index);
        if (h.err & ERR_TIMEOUT) return fail(FSS_ERR_TIMEOUT, "a bounded device wait gave up");
        return fail(FSS_ERR_CAPACITY, "%lld tile-surfel pairs needed, capacity %lld", (long long)h.pairs_needed,
                    (long long)pair_capacity);
    }
    return FSS_OK;
}

fss_status fss_loss_l2_l1(const fss_params* params, int64_t n_pix, const void* feat, const float* rgb,
                          const void* feat_target, const float* rgb_target, float w_feat, float w_rgb, void* d_feat,
                          float* d_rgb, double* loss, fss_stream_t stream) {
    fss_status s = check_params(params);
    if (s != FSS_OK) return s;
    if (n_pix < 0) return fail(FSS_ERR_INVALID_ARG, "n_pix < 0");
    if (n_pix > 0 && (!feat || !rgb || !feat_target || !rgb_target || !d_feat || !d_rgb))
        return fail(FSS_ERR_INVALID_ARG, "NULL loss argument");
    if (!loss) return fail(FSS_ERR_INVALID_ARG, "loss is NULL");
    if (misaligned16(feat) || misaligned16(feat_target) || misaligned16(d_feat))
        return fail(FSS_ERR_INVALID_ARG, "feature buffers must be 16-byte aligned");
    cudaError_t e = launch_loss(n_pix, params->C, params->out_dtype, feat, rgb, feat_target, rgb_target, w_feat, w_rgb,
                                d_feat, d_rgb, loss, num_sms_current(), reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "loss");
    return FSS_OK;
}

fss_status fss_query_labels(int64_t N, int32_t n_queries, int32_t dim, const void* f_ins, const float* means,
                            const void* f_q, const float* p_q, const float* prec_q, void* labels, int32_t out_dtype,
                            int32_t* err, fss_stream_t stream) {
    if (N < 0 || N > (int64_t)INT32_MAX * 128) return fail(FSS_ERR_UNSUPPORTED, "N %lld out of range", (long long)N);
    if (n_queries < 16 || n_queries > 256 || n_queries % 16)
        return fail(FSS_ERR_UNSUPPORTED, "n_queries %d must be a multiple of 16 in [16,256]", n_queries);
    if (dim < 16 || dim > 128 || dim % 16)
        return fail(FSS_ERR_UNSUPPORTED, "dim %d must be a multiple of 16 in [16,128]", dim);
    if (out_dtype != FSS_F32 && out_dtype != FSS_BF16) return fail(FSS_ERR_INVALID_ARG, "out_dtype %d", out_dtype);
    if (!err || !f_q || !p_q || !prec_q) return fail(FSS_ERR_INVALID_ARG, "NULL query argument or err");
    if (N > 0 && (!f_ins || !means || !labels)) return fail(FSS_ERR_INVALID_ARG, "NULL Gaussian argument");
    if (misaligned16(f_ins) || misaligned16(f_q) || misaligned16(labels))
        return fail(FSS_ERR_INVALID_ARG, "f_ins, f_q and labels must be 16-byte aligned");
    cudaError_t e = launch_query_labels(N, n_queries, dim, f_ins, means, f_q, p_q, prec_q, labels,
                                        out_dtype == FSS_BF16, err, num_sms_current(),
                                        reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "query_labels");
    return FSS_OK;
}

const char* fss_last_error(void) { return g_err.c_str(); }

fss_status fss_test_hold_scan(int32_t hold) {
    const cudaError_t e = set_hold_scan(hold != 0);
    return e == cudaSuccess ? FSS_OK : cuda_fail(e, "fss_test_hold_scan");
}

fss_status fss_set_kernel_events(void* const* events, int32_t n_events) {
    if (n_events < 0 || (n_events > 0 && !events)) return fail(FSS_ERR_INVALID_ARG, "events is NULL or n_events < 0");
    for (int32_t k = 0; k < n_events; ++k)
        if (!events[k]) return fail(FSS_ERR_INVALID_ARG, "event %d is NULL", k);
    g_mark_ev = n_events ? reinterpret_cast<cudaEvent_t*>(const_cast<void**>(events)) : nullptr;
    g_mark_n = n_events;
    g_mark_k = 0;
    return FSS_OK;
}

}  // extern "C"
