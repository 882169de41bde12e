// Kernel declarations shared between the translation units of the library.
#pragma once

#include "fss_internal.cuh"

namespace fss {

// Per-tile depth sort: CTAs of SORT_THREADS threads and lists of up to
// SORT_CAP keys in shared memory (8 KB), so that eight CTAs fit on an SM and
// the 1,200 tiles of a 640 x 480 frame sort in one wave
constexpr int SORT_THREADS = 128;
constexpr int SORT_CAP = 1024;

// Measurement hook (fss_set_kernel_events): called right after every kernel
// launch; records the calling thread's next caller-supplied event, if any,
// on the launch stream.
void kernel_mark(cudaStream_t s);
// True while that hook has events left: the timed launches then stay in the
// launch stream, one after another.
bool kernel_marks_armed();

// A second stream of the calling thread on the current device, with a fork
// and a join event, for work that may overlap the launch stream `s`.  False
// when there is none (not created while `s` is being captured, or creation
// failed): the caller then stays in `s`.
bool side_stream(cudaStream_t s, cudaStream_t& side, cudaEvent_t& fork, cudaEvent_t& join);

__global__ void k_project(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                          const float* __restrict__ means, const float* __restrict__ scales,
                          const float* __restrict__ quats, const float* __restrict__ opac, float4* __restrict__ rec,
                          BinRec* __restrict__ binrec, uint32_t* __restrict__ count, uint32_t* __restrict__ tile_cnt,
                          uint32_t* __restrict__ vis_list, uint32_t* __restrict__ wide_list,
                          uint32_t* __restrict__ unb_list, int32_t* __restrict__ splat_slot,
                          int32_t* __restrict__ slot_surf, Status* __restrict__ st);
cudaError_t set_hold_scan(int hold);  // fss_test_hold_scan
__global__ void k_emit(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                       const BinRec* __restrict__ binrec, const uint32_t* __restrict__ vis_list,
                       const uint32_t* __restrict__ wide_list, const uint32_t* __restrict__ unb_list,
                       uint32_t* __restrict__ cursor, int2* __restrict__ ranges, int32_t* __restrict__ order,
                       uint32_t* __restrict__ list, const float* __restrict__ means, const float* __restrict__ scales,
                       const float* __restrict__ quats, float4* __restrict__ rec, Status* __restrict__ st,
                       int max_lines);
__global__ void k_tile_sort(const __grid_constant__ Cams cams, const __grid_constant__ RParams P,
                            const float4* __restrict__ rec, const BinRec* __restrict__ binrec,
                            const int2* __restrict__ ranges, uint32_t* __restrict__ list,
                            const uint32_t* __restrict__ unb_list, uint64_t* __restrict__ scratch,
                            uint32_t* __restrict__ masks, const Status* __restrict__ st);

// forward render arguments (one struct so the template instances share a
// signature)
struct FwdArgs {
    const float4* rec;
    const BinRec* binrec;
    const int2* ranges;
    const uint32_t* list;
    const uint32_t* masks;  // per pair: warps of its tile that the footprint reaches
    const float* rgb;
    const void* feats;
    void* out_feat;
    float* out_rgb;
    float* out_T;
    int32_t* out_ids;
    int32_t* saved_pos;  // [pix, K]
    float* saved_w;      // [pix, K]
    int32_t* saved_nstop;  // [pix]
    Status* st;
    int persistent;
};

// training loss fused into the Top-K forward (its LOSS instances): the
// definition and arithmetic of k_loss, on F as stored in the feature type
struct LossOut {
    const void* Ft;     // [pix, C] target features, feature type
    const float* rgbt;  // [pix, 3]
    void* dF;           // [pix, C] dL/dF, feature type
    float* drgb;        // [pix, 3] dL/drgb
    double* loss;       // one double, zeroed before the launch
    float sf;           // 2 w_f / (n C): dL/dF = sf (F - F_t)
    float lf;           // w_f / (n C): the feature term's weight on sum (F - F_t)^2
    float sc;           // w_c / (3 n): dL/drgb = sc sign(rgb - rgb_t), and the weight on sum |rgb - rgb_t|
};

// the depth sort run by the Top-K forward on its own tile (its SORT
// instances; sort_tile in sort.cuh): the workspace regions the sort kernel takes
struct SortIn {
    const BinRec* binrec;
    uint32_t* list;  // sorted in place
    uint32_t* masks;
    const uint32_t* unb_list;
    uint64_t* scratch;
};

// sensor outputs of the forward render, each may be NULL, the fused loss
// (loss.loss NULL: none) and the fused sort (sort.list NULL: none).  A kernel
// parameter of its own: a larger FwdArgs costs the main Top-K instance
// register spills.
struct AuxOut {
    float* depth;      // [pix] sum w z_hit
    float* depth_med;  // [pix] z_hit where T first drops below 1/2, else 0
    float* normal;     // [pix, 3] sum w n, camera-space normals facing the camera
    int32_t* label;    // [pix] argmax over the channels of the rendered features, -1 if none blended
    LossOut loss;
    SortIn sort;
    __host__ __device__ bool any() const { return depth || depth_med || normal || label; }
};

// launchers (defined in render_fwd.cu / render_bwd.cu); return a cudaError_t
cudaError_t launch_render_forward(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                                  cudaStream_t stream);
// the full-accumulation kernel (K = 0), in render_full.cu, and the Top-K kernel
// per feature type, in render_topk_f32.cu / render_topk_bf16.cu
cudaError_t launch_render_full(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                               cudaStream_t stream);
cudaError_t launch_render_topk_f32(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                                   cudaStream_t stream);
cudaError_t launch_render_topk_bf16(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                                    cudaStream_t stream);

struct BwdArgs {
    const float4* rec;
    const BinRec* binrec;
    const int2* ranges;
    const uint32_t* list;
    const uint32_t* masks;
    const float* rgb;
    const void* feats;
    const int32_t* saved_pos;
    const float* saved_w;
    const int32_t* saved_nstop;
    const float* out_T;
    const void* d_feat;
    const float* d_rgb;
    const float* d_T;
    float* dots;        // [pix, K] c_i . dL/dF for the selected surfels
    float* grad_item;   // [n_cams * N, GRAD_STRIDE] per (view, slot)
    float* feat_acc;    // [N, C] f32 accumulation per slot
    const int32_t* splat_slot;  // [N]
    const int32_t* slot_surf;   // [N] surfel of each slot
    const float* means;
    const float* scales;
    const float* quats;
    const float* opac;
    int persistent;  // tile kernels pull tiles from the status block's queues
    float* g_means;
    float* g_scales;
    float* g_quats;
    float* g_opac;
    float* g_rgb;
    void* g_feat;
    Status* st;
};

// sh: spherical-harmonic colour coefficients [N, B, 3] (colour mode SH; a.rgb
// then points at the forward's item colours), else NULL
cudaError_t launch_render_backward(const Cams& cams, const RParams& P, const BwdArgs& a, const float* sh, int num_sms,
                                   cudaStream_t stream);

// query-guided instance labels (query.cu): l_ins [N, nq] (F32 or BF16) from
// BF16 f_ins [N, dim] and f_q [nq, dim]; nq in {16, 32, ..., 256}, dim in
// {16, 32, ..., 128}; *err set to 1 if a bounded wait on the tensor cores expired
size_t query_labels_smem(int nq, int dim);
cudaError_t launch_query_labels(int64_t N, int nq, int dim, const void* f_ins, const float* means, const void* f_q,
                                const float* p_q, const float* prec, void* out, int out_bf16, int32_t* err,
                                int num_sms, cudaStream_t stream);

// view-dependent colours (color.cu): item directions at binning, item colours
// before the forward render
cudaError_t launch_sh_dir(const Cams& cams, const RParams& P, const uint32_t* vis_list, const uint32_t* wide_list,
                          const uint32_t* unb_list, const float* means, float4* dir, const Status* st, int num_sms,
                          cudaStream_t stream);
cudaError_t launch_sh_color(const Cams& cams, const RParams& P, const uint32_t* vis_list, const uint32_t* wide_list,
                            const uint32_t* unb_list, const float4* dir, const float* coef, float* color,
                            const Status* st, int num_sms, cudaStream_t stream);

cudaError_t launch_loss(int64_t n_pix, int C, int dtype, const void* F, const float* rgb, const void* Ft,
                        const float* rgbt, float wf, float wc, void* dF, float* drgb, double* loss, int num_sms,
                        cudaStream_t s);

}  // namespace fss
