// pd_noalloc.cu — pd_process_noalloc: the chain without any device
// allocation, for callers that must not allocate.
//
// The common-mode kernels write one float per (frame, unit) that the stencil
// kernel then reads.  pd_process keeps that scratch in the context and grows
// it with cudaMalloc when a call needs more.  Here the scratch is the
// file-scope array g_cm_scratch instead, sized for kNoAllocMaxCm floats and
// present on every device that loads this library, for the life of the
// process.  Its device address is resolved by pd_create on the context's
// device (which allocates anyway); with CUDA's lazy module loading that
// lookup is also what loads this file's module and commits the array, so a
// no-allocation call made on a context's device finds the address cached and
// loads nothing.
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

// Device address of g_cm_scratch on device `dev`, which must be current
// (the first use on a device resolves and caches it).
int scratch_address(int dev, float** out, const char** why) {
    if (dev < 0 || dev >= kMaxDevices) {
        *why = "device index beyond the no-allocation table";
        return PD_ECUDA;
    }
    cudaError_t e = cudaSuccess;
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

namespace pd {

// Called by pd_create with the context's device current: resolves (and so,
// under lazy loading, loads) the scratch there.  A failure is not fatal to
// pd_create; the no-allocation call then tries again itself.
void noalloc_prepare(int dev) {
    float* p = nullptr;
    const char* why = nullptr;
    if (scratch_address(dev, &p, &why) != PD_OK) cudaGetLastError();
}

}  // namespace pd

extern "C" int pd_process_noalloc(pd_ctx* ctx, const uint16_t* frames_dev, uint32_t n_frames,
                                  uint32_t frame_base, const pd_outputs* out, void* stream) {
    const char* why = nullptr;
    int rc = pd::internal_check_process_args(ctx, frames_dev, n_frames, out, &why);
    if (rc) return pd::internal_fail(rc, why);
    // the scratch belongs to one device: the context's must be current
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != pd::internal_ctx_device(ctx))
        return pd::internal_fail(PD_EINVAL,
                                 "pd_process_noalloc: the context's device must be current");
    float* cm = out->cm;
    // (the one-kernel chain keeps its common mode on chip: no scratch, no limit)
    if (!cm && pd::internal_uses_cm_scratch(ctx)) {
        const uint64_t need = (uint64_t)n_frames * pd::internal_cm_per_frame(ctx);
        if (need > kNoAllocMaxCm)
            return pd::internal_fail(PD_EINVAL,
                                     "pd_process_noalloc: n_frames * cm_values_per_frame exceeds "
                                     "PD_NOALLOC_MAX_CM; split the call or pass out->cm");
        rc = scratch_address(dev, &cm, &why);
        if (rc) return pd::internal_fail(rc, why);
    }
    // g_cm_scratch needs no clearing: each common-mode value is written by
    // the common-mode kernel before the stencil kernel reads it.
    return pd::internal_run_sequential(ctx, frames_dev, n_frames, frame_base, out, cm,
                                       (cudaStream_t)stream);
}
