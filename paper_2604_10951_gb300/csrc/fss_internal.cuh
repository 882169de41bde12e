// Internal declarations of the sm_103a rasterizer library: device-side
// camera and parameter blocks, record layouts and the workspace layout.
// Not part of the public ABI (include/fss.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fss.h"

// Debug build with device-side index checks (compiled with
// -DFSS_CHECK_BOUNDS=1): every index that comes from device data (tile
// ranges, list entries, saved list positions, gradient slots, counters) is
// checked before use; a failed check records its site and index in the
// status block, raises ERR_BOUNDS and skips the access, so the kernel never
// faults and fss_read_status reports FSS_ERR_BOUNDS.  The workspace also
// gets a 256-byte canary after every region, checked by fss_read_status.
// Release builds compile every check away.
#ifndef FSS_CHECK_BOUNDS
#define FSS_CHECK_BOUNDS 0
#endif

namespace fss {

// ---------------------------------------------------------------------------
// launch-time constant blocks (passed by value as kernel parameters, so a
// captured CUDA graph carries them and no host->device copy is needed)
// ---------------------------------------------------------------------------
struct CamDev {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float near_plane;
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    int32_t tile_off;  // first global tile id of this view
    int64_t pix_off;   // first pixel of this view in the concatenated outputs
};

struct Cams {
    int32_t n;
    int32_t total_tiles;
    int64_t total_pix;
    const int32_t* tile_order;  // [total_tiles] tiles by descending pair count (written by k_emit), or null
    CamDev c[FSS_MAX_CAMS];
};

struct RParams {
    int32_t ts, K, bin_mode, stop_rule;
    float alpha_min, alpha_max, T_min;
    int32_t feat_dtype, out_dtype, C;
    int32_t select;  // FSS_SELECT_TOPW | FSS_SELECT_FRONT
    int32_t renorm;  // Top-K features divided by the selected weights' sum
    int32_t lowpass;   // 2DGS screen-space low-pass filter
    int32_t color_sh;  // colours per (view, surfel) item from spherical harmonics
    int32_t sh_deg;
    float bg[3];
    int64_t N;
    int64_t n_items;
    int64_t pair_cap;
};

// ---------------------------------------------------------------------------
// records
// ---------------------------------------------------------------------------
// Render record of one (view, surfel) item, 4 x float4:
//   r0 = (m0, xc), r1 = (m1, yc), r2 = (m2, det), r3 = (o, z, k2, s)
// s = 2^-e is the exact rescale applied to adj(T') (and det).
// m0..m2: rows of adj(T') (power-of-two rescaled), T' the homogeneous
// transform expressed about the local pixel origin (xc, yc); for a pixel
// point X = (x - xc, y - yc, 1): c = (m0.X, m1.X, m2.X), (u, v) = c01 / c2,
// hit depth = det / c2.
struct alignas(16) BinRec {
    float A, B, C, D, E, F;  // conic of the binning cutoff, local coordinates
    float X0, Y0, hx, hy;    // ellipse centre and half extents (local)
    float xc, yc;            // local origin (pixels)
    int16_t px0, px1, py0, py1;  // SnugBox pixel-centre range (inclusive)
    int16_t tx0, tx1, ty0, ty1;  // outer tile rectangle of the bin mode
    int32_t flags;           // BR_VISIBLE | BR_UNBOUNDED | BR_ELL | BR_LOWPASS
    float rd2;               // low-pass filter: screen disc radius^2 (pixels^2)
    int32_t pad[2];
};
static_assert(sizeof(BinRec) == 80, "BinRec layout");
// BR_ELL: the cutoff ellipse has pixels (always set without the low-pass
// filter); BR_LOWPASS: the screen disc of the low-pass filter joins it
enum { BR_VISIBLE = 1, BR_UNBOUNDED = 2, BR_ELL = 4, BR_LOWPASS = 8 };

// status block at the head of the workspace; everything from `counters` on
// is cleared at the start of each frame, `err` only by fss_read_status
struct Status {
    int32_t err;           // ERR_CAPACITY | ERR_TIMEOUT | ERR_BOUNDS
    uint32_t guards;       // check build: GUARD_WORD once the workspace canaries are written
    int64_t pairs_needed;  // pairs of the last binning (the paper's RN-Total)
    uint64_t counters[8];  // 0 evaluations, 1 contributions, 2 pixels stopped early
    uint32_t nvis;         // bounded visible items listed by k_project
    uint32_t work;         // persistent work-queue head of the forward render
    uint32_t nslot;        // surfels visible in at least one view (gradient slots)
    uint32_t work_feat;    // work-queue heads of the backward tile kernels
    uint32_t work_geo;
    uint32_t nwide;        // bounded visible items spanning many tiles
    uint32_t scan_ticket;  // k_emit: the first CTA to take it scans the tile counts
    uint32_t scan_done;    // ... and sets this (release) once the ranges and cursors are written
    uint32_t unb_cnt[FSS_MAX_CAMS];  // unbounded items per view
    uint32_t bounds_site;            // check build: first failed index check (BoundsSite), else 0
    uint32_t pad4;
    int64_t bounds_index;            // ... and the index it refused
};
enum { ERR_CAPACITY = 1, ERR_TIMEOUT = 2, ERR_BOUNDS = 4 };

// sites of the index checks of the check build (names in api.cu)
enum BoundsSite : uint32_t {
    SITE_NONE = 0,
    SITE_TILE,        // a tile id from binning (tile counts, emit cursors)
    SITE_VIS_LIST,    // a slot of the visible / wide / unbounded item lists
    SITE_SLOT,        // a gradient slot or the surfel of one
    SITE_RANGE,       // a tile's range of the pair list
    SITE_ITEM,        // a (view, surfel) item read from the pair list
    SITE_SORT_SCRATCH,  // the radix sort's global scratch
    SITE_LIST_POS,    // a saved list position of a selected entry
    SITE_FEAT_ROW,    // a feature row id
    SITE_COUNT
};

// Check build: true if 0 <= i < n; otherwise records the site and index in
// the status block (the first failure only), raises ERR_BOUNDS and returns
// false so that the caller skips the access.  Release build: always true.
__device__ __forceinline__ bool in_bounds(Status* st, BoundsSite site, int64_t i, int64_t n) {
#if FSS_CHECK_BOUNDS
    if (i >= 0 && i < n) return true;
    if (atomicCAS(&st->bounds_site, 0u, (uint32_t)site) == 0u) st->bounds_index = i;
    atomicOr(&st->err, ERR_BOUNDS);
    return false;
#else
    (void)st; (void)site; (void)i; (void)n;
    return true;
#endif
}
// a condition that only the check build tests (true in release builds)
#if FSS_CHECK_BOUNDS
#define FSS_CHECKED(cond) (cond)
#else
#define FSS_CHECKED(cond) true
#endif

// a tile's range [x, y) of a pair list of capacity cap; an invalid range
// becomes empty (check build)
__device__ __forceinline__ int2 checked_range(const int2* ranges, int t, int64_t cap, Status* st) {
    int2 rg = ranges[t];
#if FSS_CHECK_BOUNDS
    if (!(rg.x >= 0 && rg.x <= rg.y && (int64_t)rg.y <= cap)) {
        in_bounds(st, SITE_RANGE, rg.y > cap ? (int64_t)rg.y : (int64_t)rg.x, rg.x < 0 ? 0 : cap + 1);
        rg = make_int2(0, 0);
    }
#else
    (void)cap; (void)st;
#endif
    return rg;
}
constexpr size_t STATUS_CLEAR_OFF = 16;  // offsetof(Status, counters)
static_assert(STATUS_CLEAR_OFF == 16 && sizeof(int32_t) + sizeof(uint32_t) + sizeof(int64_t) == 16,
              "err, guards and pairs_needed precede the per-frame part of the status block");
// check build: a 256-byte canary of GUARD_BYTE after every workspace region
constexpr size_t GUARD_BYTES = FSS_CHECK_BOUNDS ? 256 : 0;
constexpr unsigned char GUARD_BYTE = 0xA5;
constexpr uint32_t GUARD_WORD = 0xA5A5A5A5u;

// ---------------------------------------------------------------------------
// workspace layout (host computed, identical for every call of a frame)
// ---------------------------------------------------------------------------
// Per-tile pair counters (the emit cursors after the scan) sit one 32-byte
// sector apart: every pair of the frame adds to one of them, and packed 32
// to an L2 line the adds of the whole GPU queued on a few dozen lines.
constexpr int TC_STRIDE = 8;

enum Region {
    REG_STATUS = 0,
    REG_REC = 1,
    REG_BINREC = 2,
    REG_COUNT = 3,
    REG_RANGES = 4,
    REG_LIST = 5,
    REG_COUNTERS = 6,
    REG_TILECNT = 7,
    REG_SORTTMP = 8,
    REG_GRAD_ITEM = 9,
    REG_FEAT_ACC = 10,
    REG_DOTS = 11,
    REG_VIS = 12,
    REG_UNB = 13,
    REG_SLOT = 14,   // int32 [N]: gradient slot of each surfel, -1 if culled in every view
    REG_WIDE = 15,   // uint32 [items]: visible items spanning many tiles
    REG_MASK = 16,   // uint32 [pair_capacity]: per sorted pair, the warps of its tile it reaches
    REG_SLOT_SURF = 17,  // int32 [N]: surfel of each gradient slot
    REG_DIR = 18,    // float4 [items] (spherical-harmonic colours only): unit direction from the camera, 1/distance
    REG_COLOR = 19,  // float [items, 3] (spherical-harmonic colours only): each visible item's colour
    REG_ORDER = 20,  // int32 [tiles]: the order the tile kernels take tiles in (heavy first)
    REG_COUNT_ALL
};

struct Layout {
    size_t off[REG_COUNT_ALL];
    size_t size[REG_COUNT_ALL];
    size_t total;
};

constexpr int GRAD_STRIDE = 16;  // floats per item in the geometric gradient buffer

// view that owns global tile t (views are laid out by increasing tile_off)
__device__ __forceinline__ int view_of_tile(const Cams& cams, int t) {
    int lo = 0, hi = cams.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams.c[mid].tile_off <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace fss
