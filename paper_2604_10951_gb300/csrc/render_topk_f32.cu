// Top-K forward render instances for FP32 feature rows.
#include "render_topk.cuh"

namespace fss {

cudaError_t launch_render_topk_f32(const Cams& cams, const RParams& P, const FwdArgs& a, const AuxOut& x, int num_sms,
                                   cudaStream_t stream) {
    return launch_topk_dtype<float>(cams, P, a, x, num_sms, stream);
}

}  // namespace fss
