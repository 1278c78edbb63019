// pd_noalloc.cu — pd_process_noalloc: the chain without any device
// allocation, for callers that must not allocate.
//
// The common-mode kernels write one float per (frame, unit) that the stencil
// kernel then reads.  pd_process keeps that scratch in the context and grows
// it with cudaMalloc when a call needs more.  Here the scratch is the
// file-scope array g_cm_scratch instead, sized for kNoAllocMaxCm floats and
// present on every device that loads this library, for the life of the
// process.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "pd.h"
#include "pd_internal.cuh"

namespace {

constexpr uint32_t kNoAllocMaxCm = PD_NOALLOC_MAX_CM;  // floats (4 MiB)
constexpr int kMaxDevices = 64;

// Device-side scratch of the common-mode values.  In host code this name is
// only a stand-in for the symbol: its device address comes from
// cudaGetSymbolAddress, taken once per device below.
static __device__ __align__(256) float g_cm_scratch[kNoAllocMaxCm];

std::mutex g_mu;
float* g_ptr[kMaxDevices] = {};

// Device address of g_cm_scratch on the current device (first use on a
// device resolves and caches it).
int scratch_address(float** out, const char** why) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        *why = "no usable current device";
        return PD_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cm_scratch);
        if (e != cudaSuccess || !p) {
            *why = "cudaGetSymbolAddress failed for the common-mode scratch";
            return PD_ECUDA;
        }
        g_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_ptr[dev];
    return PD_OK;
}

}  // namespace

extern "C" int pd_process_noalloc(pd_ctx* ctx, const uint16_t* frames_dev, uint32_t n_frames,
                                  uint32_t frame_base, const pd_outputs* out, void* stream) {
    const char* why = nullptr;
    int rc = pd::internal_check_process_args(ctx, frames_dev, n_frames, out, &why);
    if (rc) return pd::internal_fail(rc, why);
    float* cm = out->cm;
    if (!cm) {
        const uint64_t need = (uint64_t)n_frames * pd::internal_cm_per_frame(ctx);
        if (need > kNoAllocMaxCm)
            return pd::internal_fail(PD_EINVAL,
                                     "pd_process_noalloc: n_frames * cm_values_per_frame exceeds "
                                     "PD_NOALLOC_MAX_CM; split the call or pass out->cm");
        rc = scratch_address(&cm, &why);
        if (rc) return pd::internal_fail(rc, why);
    }
    // g_cm_scratch needs no clearing: each common-mode value is written by
    // the common-mode kernel before the stencil kernel reads it.
    return pd::internal_run_sequential(ctx, frames_dev, n_frames, frame_base, out, cm,
                                       (cudaStream_t)stream);
}
