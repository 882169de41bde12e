// Forward render dispatch: the full-accumulation kernel (K = 0, render_full.cu)
// or the Top-K kernel (render_topk.cuh, one translation unit per feature type).
#include "fss_internal.cuh"
#include "kernels.cuh"

namespace fss {

cudaError_t launch_render_forward(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                                  cudaStream_t stream) {
    if (P.K == 0) return launch_render_full(cams, P, a, x, num_sms, stream);
    if (P.feat_dtype == FSS_BF16) return launch_render_topk_bf16(cams, P, a, x, num_sms, stream);
    return launch_render_topk_f32(cams, P, a, x, num_sms, stream);
}

}  // namespace fss
