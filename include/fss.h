/*
 * fss.h -- C ABI of the GB300 (sm_103a) 2D Gaussian Splatting feature
 * rasterizer with Precise Tile Intersection and Top-K Hard Selection
 * (Fast-SegSim, arXiv 2604.10951).
 *
 * All device memory is owned by the caller.  The library allocates nothing:
 * every entry point works inside a caller-provided `workspace` (size from
 * fss_workspace_size) and caller-provided outputs.  The one exception is
 * fss_forward_static, which uses a fixed static device array instead.  Every
 * other compute call is asynchronous on the given CUDA stream (`fss_stream_t`
 * is the same type as cudaStream_t; NULL means the legacy default stream) and
 * can be captured in a CUDA graph.  Only fss_read_status and
 * fss_forward_static synchronise with the host.
 *
 * Conventions shared by all calls:
 *   - surfel parameters are float32, row-major, N rows:
 *       means [N,3] world position p_i; scales [N,2] (r_u, r_v) > 0 (already
 *       activated); quats [N,4] (w,x,y,z), any non-zero length (normalised
 *       inside); opac [N] opacity o_i in [0,1] (already activated);
 *       rgb [N,3]; feats [N,C] (float32 or bfloat16, params->feat_dtype)
 *     (Sec. 3.1, Eq. 1: p(u) = p_i + r_u t_u u + r_v t_v v, t_u and t_v the
 *     first two columns of R(q)).
 *   - cameras: OpenCV pinhole (x right, y down, z forward); viewmat is the
 *     row-major 3x4 world->camera [R | t]; pixel (px,py) is sampled at its
 *     centre (px+0.5, py+0.5).  Up to FSS_MAX_CAMS views per call; view v
 *     owns pixels [pix_off(v), pix_off(v) + H_v*W_v) of every per-pixel
 *     output, pix_off(v) = sum over u < v of H_u*W_u (views concatenated).
 *   - per-pixel outputs are row-major [H, W, ...] per view.
 *   - the workspace layout depends on (params->tile_size, K, C, feat dtype,
 *     cameras, N, pair_capacity): pass identical values to every call that
 *     shares a workspace.
 *
 * Errors: a call returns FSS_ERR_INVALID_ARG or FSS_ERR_UNSUPPORTED without
 * launching anything when its arguments are bad, FSS_ERR_CUDA when a launch
 * fails; fss_last_error() then holds a message for the calling thread.
 * Errors found on the device (too many tile-surfel pairs, a bounded wait
 * that ran out) are recorded in the workspace, make later kernels of the
 * same frame do nothing, and are returned by fss_read_status.
 *
 * Check build: the library compiled with -DFSS_CHECK_BOUNDS=1
 * (libfss_check.so) checks, on the device, every index it takes from device
 * data (tile ranges, pair-list entries, saved Top-K list positions,
 * gradient slots, list counters) before using it.  A failed check skips the
 * access, records its site and index, and makes fss_read_status return
 * FSS_ERR_BOUNDS; nothing traps.  Its workspace (a larger
 * fss_workspace_size) also holds a 256-byte canary after every region,
 * written by fss_project_bin and verified by fss_read_status.  The API and
 * results are otherwise those of the release build.
 *
 * Side streams: an eager (not captured) fss_render_backward may run part of
 * its work in a second stream that the library creates once per calling
 * thread and device, joined to `stream` before the call returns (also on
 * errors); the thread's streams are destroyed when it exits.
 */
#ifndef FSS_H
#define FSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fss_stream_t; /* == cudaStream_t */

typedef enum {
    FSS_OK = 0,
    FSS_ERR_INVALID_ARG = 1,
    FSS_ERR_UNSUPPORTED = 2,
    FSS_ERR_CAPACITY = 3, /* more tile-surfel pairs than pair_capacity */
    FSS_ERR_CUDA = 4,
    FSS_ERR_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    FSS_ERR_BOUNDS = 6    /* check build only (FSS_CHECK_BOUNDS): a device index check or a workspace
                             canary failed; the refused access was skipped */
} fss_status;

enum { FSS_BIN_AABB = 0, FSS_BIN_SNUG = 1, FSS_BIN_ACCU = 2 };
enum { FSS_STOP_TMIN = 0, FSS_STOP_EXACT_TOPK = 1 };
enum { FSS_F32 = 0, FSS_BF16 = 1 };

#define FSS_MAX_CAMS 64
#define FSS_MAX_K 32

typedef struct {
    float fx, fy, cx, cy;  /* pinhole intrinsics in pixels */
    int32_t width, height; /* image size in pixels, 1..16384 */
    float viewmat[12];     /* row-major 3x4 world->camera [R | t] */
    float near_plane;      /* hits at camera depth <= near_plane are skipped */
} fss_camera;

typedef struct {
    int32_t tile_size;  /* 8, 16 or 32 pixels per tile side */
    int32_t K;          /* 0: full accumulation (Eq. 2); 1..32: Top-K (Eq. 7) */
    int32_t bin_mode;   /* FSS_BIN_AABB | FSS_BIN_SNUG | FSS_BIN_ACCU (Sec. 3.2) */
    int32_t stop_rule;  /* FSS_STOP_TMIN | FSS_STOP_EXACT_TOPK */
    float alpha_min;    /* contributions below are skipped (default 1/255) */
    float alpha_max;    /* alpha clamp (default 0.99) */
    float T_min;        /* stop before transmittance would fall below (1e-4) */
    int32_t feat_dtype; /* FSS_F32 | FSS_BF16: storage of feats and of their gradient */
    int32_t out_dtype;  /* FSS_F32 | FSS_BF16: storage of the rendered features */
    int32_t C;          /* feature channels: multiple of 4 (F32) / 8 (BF16), 4..512 */
    float bg_rgb[3];    /* background colour added as T_final * bg */
    int32_t schedule;   /* FSS_SCHED_GRID: one CTA per tile; FSS_SCHED_PERSISTENT:
                           one wave of CTAs pulling tiles from a device work
                           queue (balances views of mixed size) */
    int32_t select;     /* K > 0: FSS_SELECT_TOPW, the K largest blending weights
                           (Eq. 7); FSS_SELECT_FRONT, the first K contributors
                           in depth order (the other reading of the selection set) */
    int32_t renorm;     /* K > 0: 0 = Eq. 7 as printed (no normalisation); 1 = divide
                           the Top-K feature sum by the selected weights' sum, so the
                           selected surfels' weights add up to 1 (a variant; K = 0
                           rejects it) */
    int32_t color_mode; /* FSS_COLOR_RGB: the rgb argument of the render calls is a
                           per-surfel colour [N, 3]; FSS_COLOR_SH: it holds
                           view-dependent colour coefficients [N, (sh_degree+1)^2, 3]
                           of real spherical harmonics (Sec. 3.1's view-dependent
                           colour): c = max(0, sum_b k_b Y_b(d) + 1/2), d the unit
                           direction from the camera centre to the surfel centre,
                           Y_b without the Condon-Shortley sign, b = l^2 + l + m;
                           the backward's g_rgb then has the coefficients' shape and
                           g_means gains the direction term */
    int32_t sh_degree;  /* 0..3 (FSS_COLOR_SH) */
    int32_t lowpass;    /* 1: the 2DGS screen-space low-pass filter, alpha = o exp(-rho/2)
                           with rho = min(u^2 + v^2, 2 |x - c|^2), c the projected
                           centre (the screen term takes the centre's depth); the
                           binning adds the screen disc 2 |x - c|^2 <= k^2 */
} fss_params;

enum { FSS_SCHED_GRID = 0, FSS_SCHED_PERSISTENT = 1 };
enum { FSS_SELECT_TOPW = 0, FSS_SELECT_FRONT = 1 };
enum { FSS_COLOR_RGB = 0, FSS_COLOR_SH = 1 };

/* Fills the defaults listed above (tile 16, K 8, ACCU, TMIN, F32, C 16, grid, TOPW, no renormalisation). */
fss_status fss_default_params(fss_params *params);

/* Bytes of device workspace needed for these cameras, N surfels and at most
 * `pair_capacity` tile-surfel pairs (the paper's RN-Total, Table 2). */
fss_status fss_workspace_size(const fss_params *params, const fss_camera *cams, int32_t n_cams,
                              int64_t N, int64_t pair_capacity, size_t *bytes);

/* Bytes of the `saved` buffer that fss_render_forward fills for the
 * backward pass (per pixel: Top-K list positions and weights, traversal
 * length). */
fss_status fss_saved_size(const fss_params *params, const fss_camera *cams, int32_t n_cams, size_t *bytes);

/*
 * Projection and Precise Tile Intersection binning (Sec. 3.2).
 * Per surfel and view: the homogeneous transform T (x' = T u), its
 * adjugate (ray-splat intersection), the opacity-aware cutoff
 * k^2 = 2 ln(o / alpha_min), the screen conic of the cutoff disc, its tight
 * box (SnugBox) and, in ACCU mode, the exact tile interval of every tile row
 * (or column, whichever span is smaller) from the quadratic
 * A x^2 + (2B y + 2D) x + (C y^2 + 2E y + F) = 0 (AccuTile).  Writes the
 * unsorted per-tile surfel lists into the workspace.  If more than
 * pair_capacity pairs are needed, records FSS_ERR_CAPACITY and the needed
 * count (see fss_read_status); the following calls then do nothing.
 * Inputs are device pointers (layout above); culled surfels (camera depth
 * <= near, o < alpha_min, seen edge-on) produce no pairs.  One CTA of the
 * emission kernel scans the per-tile counts while the others build render
 * records; their wait for its result is bounded (FSS_ERR_TIMEOUT, see
 * fss_test_hold_scan).
 */
fss_status fss_project_bin(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                           const float *means, const float *scales, const float *quats, const float *opac,
                           void *workspace, int64_t pair_capacity, fss_stream_t stream);

/*
 * Depth sort (the depth order of the compositing, Sec. 3.1): orders each tile's
 * list by (binary32 bits of the surfel centre's camera depth, surfel index),
 * a total order, so the result is deterministic.
 */
fss_status fss_sort(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                    void *workspace, int64_t pair_capacity, fss_stream_t stream);

/*
 * Forward render (Eq. 2 with Top-K Hard Selection, Eq. 7).  For every
 * pixel, front to back over its tile's sorted list: ray-splat intersection
 * (u,v), alpha = min(alpha_max, o exp(-(u^2+v^2)/2)), skip if
 * alpha < alpha_min, stop by params->stop_rule, w = alpha T, T *= 1 - alpha.
 * K = 0: F = sum_i w_i c_i over all contributors.  K > 0: F = sum over the K
 * largest w_i (ties: earlier wins; FSS_SELECT_FRONT: over the first K
 * contributors), no renormalisation unless params->renorm (then divided by
 * the sum of the selected w_i; saved weights stay unnormalised).  FSS_STOP_EXACT_TOPK stops once no
 * later surfel can enter the set (TOPW: alpha_max T <= smallest selected
 * weight; FRONT: K contributors found).
 * Device inputs: rgb [N,3] f32, feats [N,C] (feat_dtype).
 * Device outputs (any may be NULL except as noted; per view concatenated):
 *   out_feat [pix, C] in out_dtype; out_rgb [pix, 3] = sum w rgb + T bg;
 *   out_T [pix] final transmittance; out_topk_id [pix, K] surfel indices in
 *   front-to-back order, -1 padded (K > 0 only);
 *   saved: fss_saved_size bytes, required if fss_render_backward follows.
 */
fss_status fss_render_forward(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                              void *workspace, int64_t pair_capacity, const float *rgb, const void *feats,
                              void *out_feat, float *out_rgb, float *out_T, int32_t *out_topk_id,
                              void *saved, fss_stream_t stream);

/*
 * Sensor outputs of the forward render: depth images by the same alpha
 * blending as the colour (Sec. 3.5 with Eq. 2; the simulator's depth images,
 * Sec. 4.4) and normals from the tangent vectors (Sec. 3.1), each
 * [pix] or [pix, 3] float32 on the device, NULL to skip, summed over the
 * same traversed contributors as out_rgb and not renormalised:
 *   depth        sum_i w_i z_i, z_i the camera depth of the ray-surfel hit;
 *   depth_median z_i of the first contributor after which T < 1/2, else 0;
 *   normal       sum_i w_i n_i, n_i the surfel's camera-space unit normal
 *                turned to face the camera.
 * The backward pass does not differentiate them.
 */
typedef struct {
    float *depth;
    float *depth_median;
    float *normal;
    int32_t *label;     /* [pix] argmax over the C channels of the rendered features
                           (lowest channel on ties; -1 where no surfel is blended):
                           the instance mask when the features are the query labels
                           of fss_query_labels; needs no out_feat */
} fss_aux_outputs;

/* fss_render_forward plus the sensor outputs in `aux` (may be NULL); the
 * same arguments, ownership and errors.  Either call may run more than once
 * on one binning (the persistent schedule resets its tile queue first). */
fss_status fss_render_forward_aux(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                                  void *workspace, int64_t pair_capacity, const float *rgb, const void *feats,
                                  void *out_feat, float *out_rgb, float *out_T, int32_t *out_topk_id,
                                  void *saved, const fss_aux_outputs *aux, fss_stream_t stream);

/*
 * Query-guided instance labels (Sec. 3.3): for every scene Gaussian g and
 * instance query q, S = sigmoid(f_q . f_ins(g)), D = phi_q(p_g) / phi_q(p_q)
 * = exp(-1/2 d^T Sigma_q^-1 d) with d = p_g - p_q (the query's Gaussian
 * density ratio; scene Gaussians enter as points), A = S D, and
 * labels[g, :] = softmax over q of A(q, g).  The result is the per-Gaussian
 * label distribution that the render calls blend like any C = n_queries
 * feature (the paper's instance-label blending), and whose per-pixel argmax
 * fss_render_forward_aux returns as the instance mask.
 * Device inputs: f_ins [N, dim] BF16, means [N, 3] f32, f_q [n_queries, dim]
 * BF16, p_q [n_queries, 3] f32, prec_q [n_queries, 6] f32 = the entries
 * (xx, yy, zz, xy, xz, yz) of Sigma_q^-1 (symmetric positive definite).
 * Device output: labels [N, n_queries] in out_dtype (FSS_F32 | FSS_BF16).
 * n_queries: multiple of 16 in [16, 256]; dim: multiple of 16 in [16, 128];
 * f_ins, f_q and labels 16-byte aligned.  The similarity logits run on the
 * tensor cores (BF16 products, FP32 sums); the rest in FP32.
 * err: device int32 that the kernel sets to 1 if a bounded wait on the
 * tensor cores expired (the caller clears and reads it; never expected).
 * Asynchronous on `stream`; the caller owns every buffer.  Errors:
 * FSS_ERR_UNSUPPORTED for sizes out of range, FSS_ERR_INVALID_ARG for NULL
 * or misaligned pointers and bad dtypes, FSS_ERR_CUDA for launch failures.
 */
fss_status fss_query_labels(int64_t N, int32_t n_queries, int32_t dim, const void *f_ins, const float *means,
                            const void *f_q, const float *p_q, const float *prec_q, void *labels, int32_t out_dtype,
                            int32_t *err, fss_stream_t stream);

/*
 * Backward render: vector-Jacobian product of fss_render_forward for the
 * upstream gradients d_feat [pix, C] (out_dtype), d_rgb [pix, 3] f32 and
 * d_T [pix] f32 (may be NULL).  Replays each pixel back to front from the
 * saved traversal length and final transmittance; the Top-K set, skips,
 * stops and clamps are held fixed.  Outputs (overwritten, device):
 *   g_means [N,3], g_scales [N,2], g_quats [N,4], g_opac [N], g_rgb [N,3]
 *   (float32) and g_feat [N,C] (feat_dtype; FP32 accumulation inside).
 * Gradients are summed over all views of the call.
 * Stream use: outside a graph capture, with K > 0 and g_feat given, the
 * feature-gradient output pass runs in a second stream owned by the library
 * (one per calling thread and device), forked from `stream` after the work
 * it needs and joined back into `stream` before the call returns, so
 * ordering on `stream` is as if everything ran there.  A call captured into
 * a graph uses `stream` alone.
 */
fss_status fss_render_backward(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                               void *workspace, int64_t pair_capacity,
                               const float *means, const float *scales, const float *quats, const float *opac,
                               const float *rgb, const void *feats, const void *saved, const float *out_T,
                               const void *d_feat, const float *d_rgb, const float *d_T,
                               float *g_means, float *g_scales, float *g_quats, float *g_opac, float *g_rgb,
                               void *g_feat, fss_stream_t stream);

/*
 * Synchronises `stream`, then reports device-side errors of the frames
 * processed in `workspace`: FSS_ERR_CAPACITY (with *num_pairs = the number
 * of pairs needed), FSS_ERR_TIMEOUT, or FSS_OK (with *num_pairs = pairs
 * used).  Clears the error flags.  `num_pairs` may be NULL.
 */
fss_status fss_read_status(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                           void *workspace, int64_t pair_capacity, int64_t *num_pairs, fss_stream_t stream);

/*
 * Loss of the forward+backward workload and its gradient in one pass:
 *   L = w_feat * mean((F - F_t)^2) + w_rgb * mean(|rgb - rgb_t|)
 * over n_pix pixels (feature L2 standing in for the segmentation losses,
 * RGB L1 as in the photometric loss, Sec. 3.5).  Device inputs: feat and
 * feat_target [n_pix, C] in params->out_dtype, rgb and rgb_target [n_pix,3]
 * f32.  Device outputs: d_feat [n_pix, C] (out_dtype) and d_rgb [n_pix, 3]
 * ready for fss_render_backward, and *loss (one double, overwritten).
 */
fss_status fss_loss_l2_l1(const fss_params *params, int64_t n_pix, const void *feat, const float *rgb,
                          const void *feat_target, const float *rgb_target, float w_feat, float w_rgb,
                          void *d_feat, float *d_rgb, double *loss, fss_stream_t stream);

/*
 * fss_render_forward followed by fss_loss_l2_l1 on its outputs, in one call:
 * the same forward arguments, then the loss's target, weights and outputs,
 * over the n_pix pixels of all cameras (pixel order of the outputs).
 * out_feat, out_rgb and every loss argument are required; feat_target and
 * d_feat are 16-byte aligned, in params->out_dtype.  With the plain Top-K
 * selection (0 < K <= 8, not FSS_SELECT_FRONT, no low-pass filter) and
 * out_dtype == feat_dtype, the loss is evaluated inside the forward kernel
 * on each pixel's feature chunk as it is stored, so F is not read back:
 * d_feat and d_rgb equal those of the two separate calls bit for bit and
 * *loss differs by the summation order only.  Otherwise the loss kernel runs
 * after the render.  Errors as for the two calls.
 */
fss_status fss_render_forward_loss(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                                   void *workspace, int64_t pair_capacity, const float *rgb, const void *feats,
                                   void *out_feat, float *out_rgb, float *out_T, int32_t *out_topk_id,
                                   void *saved, const void *feat_target, const float *rgb_target, float w_feat,
                                   float w_rgb, void *d_feat, float *d_rgb, double *loss, fss_stream_t stream);

/*
 * fss_sort followed by fss_render_forward_loss, in one call: the same
 * arguments as fss_render_forward_loss, on a workspace that fss_project_bin
 * has just filled (unsorted tile lists).  Where the loss runs inside the
 * render kernel (the conditions above), each CTA of that kernel first sorts
 * its own tile's list (the same order and warp masks as fss_sort, written to
 * the workspace for the backward pass), so the sort needs no launch of its
 * own; otherwise the sort kernel runs first.  Outputs, workspace contents
 * and errors as for the two calls.
 */
fss_status fss_sort_render_forward_loss(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                                        void *workspace, int64_t pair_capacity, const float *rgb,
                                        const void *feats, void *out_feat, float *out_rgb, float *out_T,
                                        int32_t *out_topk_id, void *saved, const void *feat_target,
                                        const float *rgb_target, float w_feat, float w_rgb, void *d_feat,
                                        float *d_rgb, double *loss, fss_stream_t stream);

/*
 * Size of the device scratch array behind fss_forward_static: 64 MiB per
 * device, reserved when the library's module loads on that device.
 */
#define FSS_STATIC_SCRATCH_BYTES (64u << 20)

/*
 * fss_forward_static -- a forward frame that allocates nothing and needs no
 * caller workspace.  The paper has no counterpart: this is a convenience of
 * this library's C ABI.
 *
 * Who it is for: callers that cannot hand the library device memory at call
 * time.  Examples are a plain C host program with no device allocator of its
 * own; a real-time loop where cudaMalloc/cudaFree are not acceptable, since
 * cudaFree waits for the whole device; and a process whose device memory is
 * already fully reserved by another framework's pool.  Such a caller provides
 * only the surfel inputs and the outputs.
 *
 * What it does: fss_project_bin, fss_sort and fss_render_forward, then
 * fss_read_status, with the same arguments, on a workspace inside a
 * file-scope device array of FSS_STATIC_SCRATCH_BYTES.  The outputs equal
 * those calls' outputs on a caller workspace.  The call returns after
 * `stream` has finished the frame.  Results: FSS_OK (with *num_pairs = pairs
 * used; num_pairs may be NULL); FSS_ERR_CAPACITY (with *num_pairs = pairs
 * needed; retry with a larger pair_capacity); FSS_ERR_INVALID_ARG or
 * FSS_ERR_UNSUPPORTED for bad arguments or a frame over the limit below,
 * before anything is launched; FSS_ERR_CUDA when a CUDA call fails;
 * FSS_ERR_TIMEOUT as fss_read_status reports it; FSS_ERR_BOUNDS from the
 * check build only.
 *
 * Limit: a frame whose fss_workspace_size(params, cams, n_cams, N,
 * pair_capacity) exceeds FSS_STATIC_SCRATCH_BYTES is rejected with
 * FSS_ERR_UNSUPPORTED before anything is launched.  About 64 + 80 + 20 bytes
 * per (surfel, view), 64 per (surfel, view) and 4 C per surfel for the
 * gradient regions, 4 K per pixel, and 20 bytes per pair must fit.
 *
 * Set-up: the first call on each device looks up the array's address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * life of the process.  Make that first call before any stream capture.
 * A device reset (cudaDeviceReset) reloads the module at another address:
 * it is not supported while this library is in use, for this call and for
 * the library's per-thread side streams.
 *
 * Sharing: all calls on one device share the one array, so calls that
 * overlap in time race and corrupt each other's frames.  Overlap comes from
 * other streams or other host threads.  Serialise them, e.g. one stream
 * and one thread.  A frame's `saved` buffer stays valid.  Running
 * fss_render_backward on it needs the workspace, which lives in the static
 * array and is not exposed; use a caller workspace when gradients are
 * needed.
 */
fss_status fss_forward_static(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                              int64_t pair_capacity, const float *means, const float *scales,
                              const float *quats, const float *opac, const float *rgb, const void *feats,
                              void *out_feat, float *out_rgb, float *out_T, int32_t *out_topk_id, void *saved,
                              int64_t *num_pairs, fss_stream_t stream);

/*
 * Measurement hook (the paper has no counterpart): after this call, the
 * next n_events kernels that this library launches from the calling thread
 * each record one of `events` (cudaEvent_t handles created by the caller,
 * in order) on their stream right after the launch, as external events, so
 * that they also become nodes of a captured CUDA graph.  The elapsed time
 * between consecutive events is then one kernel's duration.  n_events = 0
 * switches the hook off.  The array must stay valid while the hook is on.
 * Kernels per call: fss_project_bin 2 (project; emit, whose first CTA scans
 * the tile counts), fss_sort 1,
 * fss_render_forward 1, fss_loss_l2_l1 1, fss_render_forward_loss 1 when
 * the loss runs in the render kernel (else 2), fss_sort_render_forward_loss 1
 * when the loss runs in the render kernel (else 3), fss_render_backward 4 for Top-K
 * (clear, feature gradients, geometry replay, projection) or 3 for K = 0,
 * plus 1 when g_feat is given (feature rows).
 */
fss_status fss_set_kernel_events(void *const *events, int32_t n_events);

/*
 * Failure-detection test hook (the paper has no counterpart).  In
 * fss_project_bin one CTA of the emission kernel scans the per-tile counts
 * and publishes ranges and emission cursors with a flag; the other CTAs
 * wait for the flag with a bounded wait (about a second of sleeping
 * polls), after which they record FSS_ERR_TIMEOUT (see fss_read_status) and
 * return without emitting tiles.  With hold != 0 the scanning CTA does not
 * set the flag, so that the wait runs out; hold = 0 (the default) restores
 * normal operation.  The setting is per device and process and takes effect
 * for kernels launched after the call (which synchronises with the device).
 */
fss_status fss_test_hold_scan(int32_t hold);

/* Message of the last error returned to the calling thread ("" if none). */
const char *fss_last_error(void);

/*
 * Offset and size of a named region inside the workspace (for inspection
 * and tests).  Items are (view, surfel) pairs, item = view * N + surfel.
 * Regions:
 *   0 status block; 1 render records per item (4 x float4: adjugate rows
 *   with the local origin and det, opacity/depth/cutoff/rescale);
 *   2 binning records per item (80 bytes: conic, ellipse, pixel and tile
 *   boxes, flags); 3 tile count per item (uint32); 4 tile ranges
 *   (int32 [tiles, 2]); 5 tile lists (uint32 item ids, sorted by fss_sort);
 *   6 counters (uint64 [8], inside the status block: evaluations,
 *   contributions); 7 per-tile pair counts, then emission cursors (uint32,
 *   one per 32-byte sector);
 *   8 sort scratch (2 x uint64 per pair); 9 geometric gradient rows
 *   (float [views, N, 16]); 10 feature gradient accumulators (float [N, C]);
 *   11 per-(pixel, k) dot products (float [pixels, K]); 12 visible item
 *   list; 13 unbounded items per view; 14 gradient slot per surfel (int32,
 *   -1 if culled in every view); 15 items spanning many tiles; 16 per-pair
 *   warp masks (uint32, written by fss_sort); 17 surfel of each gradient
 *   slot (int32); 18 unit view direction and inverse distance per item
 *   (float4, spherical-harmonic colours only); 19 colour per item (float
 *   [3], spherical-harmonic colours only); 20 tile order (int32 [tiles]:
 *   tiles by descending pair count, written by fss_project_bin; the tile
 *   kernels take tiles in this order).
 * The workspace costs 24 bytes per unit of pair_capacity.
 */
fss_status fss_workspace_region(const fss_params *params, const fss_camera *cams, int32_t n_cams, int64_t N,
                                int64_t pair_capacity, int32_t which, size_t *offset, size_t *bytes);

#ifdef __cplusplus
}
#endif
#endif /* FSS_H */
