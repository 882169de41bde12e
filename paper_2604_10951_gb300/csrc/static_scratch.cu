// fss_forward_static: the whole forward frame (projection + binning, depth
// sort, render) in a workspace that lives in a file-scope device array, so a
// call needs no device memory from the caller beyond inputs and outputs.
//
// The array is part of this translation unit's module: it is reserved when
// the module is loaded on a device (at the latest by the first call's
// cudaGetSymbolAddress) and never freed or resized.  Nothing here calls an
// allocator; the three stages are the ordinary entry points run on it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fss_internal.cuh"

namespace {

__device__ __align__(256) unsigned char g_static_ws[FSS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ws_ptr[kMaxDevices] = {};

// One cudaGetSymbolAddress per device, taken with that device current.
fss_status static_workspace(void** out, char* msg, size_t msg_len) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(msg, msg_len, "cudaGetDevice: %s", cudaGetErrorString(e));
        return FSS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(msg, msg_len, "device ordinal %d not in [0,%d)", dev, kMaxDevices);
        return FSS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ws_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || !p) {
            snprintf(msg, msg_len, "cudaGetSymbolAddress(static scratch) on device %d: %s", dev,
                     cudaGetErrorString(e));
            return FSS_ERR_CUDA;
        }
        g_ws_ptr[dev] = p;
    }
    *out = g_ws_ptr[dev];
    return FSS_OK;
}

}  // namespace

namespace fss {
fss_status set_error(fss_status s, const char* msg);
}

extern "C" fss_status fss_forward_static(const fss_params* params, const fss_camera* cams, int32_t n_cams,
                                         int64_t N, int64_t pair_capacity, const float* means,
                                         const float* scales, const float* quats, const float* opac,
                                         const float* rgb, const void* feats, void* out_feat, float* out_rgb,
                                         float* out_T, int32_t* out_topk_id, void* saved, int64_t* num_pairs,
                                         fss_stream_t stream) {
    size_t need = 0;
    fss_status s = fss_workspace_size(params, cams, n_cams, N, pair_capacity, &need);
    if (s != FSS_OK) return s;
    if (need > (size_t)FSS_STATIC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "fss_forward_static: this frame needs %zu bytes of workspace, the static scratch holds %zu "
                 "(FSS_STATIC_SCRATCH_BYTES); lower N, the views or pair_capacity, or use a caller workspace",
                 need, (size_t)FSS_STATIC_SCRATCH_BYTES);
        return fss::set_error(FSS_ERR_UNSUPPORTED, msg);
    }
    void* ws = nullptr;
    {
        char msg[256];
        if ((s = static_workspace(&ws, msg, sizeof msg)) != FSS_OK) return fss::set_error(s, msg);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The error word (the first word of the status block) persists between
    // frames; start clean (fss_project_bin clears the rest of the block, the
    // slots and the tile counts).
    size_t status_off = 0;
    if ((s = fss_workspace_region(params, cams, n_cams, N, pair_capacity, 0 /* the status block */, &status_off,
                                  nullptr)) != FSS_OK)
        return s;
    cudaError_t e = cudaMemsetAsync(static_cast<unsigned char*>(ws) + status_off, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "memset static status: %s", cudaGetErrorString(e));
        return fss::set_error(FSS_ERR_CUDA, msg);
    }
    if ((s = fss_project_bin(params, cams, n_cams, N, means, scales, quats, opac, ws, pair_capacity, stream)) != FSS_OK)
        return s;
    if ((s = fss_sort(params, cams, n_cams, N, ws, pair_capacity, stream)) != FSS_OK) return s;
    if ((s = fss_render_forward(params, cams, n_cams, N, ws, pair_capacity, rgb, feats, out_feat, out_rgb, out_T,
                                out_topk_id, saved, stream)) != FSS_OK)
        return s;
    return fss_read_status(params, cams, n_cams, N, ws, pair_capacity, num_pairs, stream);
}
