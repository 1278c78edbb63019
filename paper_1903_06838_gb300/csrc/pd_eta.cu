// pd_eta.cu — linearisation of the centre-of-mass offsets.
//
// The paper notes that the centroid of a photon's charge depends nonlinearly
// on where the photon landed and that centroids need linearising to give
// positions (section "Photon Subpixel Resolution", Fig. f and its caption).
// With photons landing uniformly inside the seed pixel, the true offset is
// u = F(d) - 1/2 where F is the cumulative distribution of the measured
// centroid d.  F is estimated per axis from single-photon hits (count == 1):
// a histogram of d over B bins spanning [-1, 1] (eta_hist_kernel), then
// F(d) = (counts below d's bin + position in the bin * the bin's count) / N.
// B is odd, so d = 0 (a photon whose neighbours all stay below the zero
// threshold: an atom of the distribution) sits in the middle of a bin and
// maps to the middle of its probability mass.
// All float arithmetic is round-to-nearest in the same order as the
// definition:  t = (d + 1) * (B * 0.5);  k = clamp(floor t);  phi = clamp(t -
// k, 0, 1);  u = (C[k] + phi * h[k]) / N - 1/2.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>

#include "pd.h"
#include "pd_internal.cuh"

struct pd_eta {
    uint32_t bins = 0;
    uint32_t* hist = nullptr;   // [2][bins] single-photon centroid counts
    uint32_t* below = nullptr;  // [2][bins + 1] counts below each bin
};

namespace {

__device__ __forceinline__ void eta_bin(float d, uint32_t bins, uint32_t* k, float* phi) {
    const float t = __fmul_rn(__fadd_rn(d, 1.0f), __fmul_rn((float)bins, 0.5f));
    const float kf = fminf(fmaxf(floorf(t), 0.0f), (float)(bins - 1));
    *k = (uint32_t)kf;
    *phi = fminf(fmaxf(__fsub_rn(t, kf), 0.0f), 1.0f);
}

__device__ __forceinline__ bool single(const pd_hit& h) {
    return h.count == 1 && isfinite(h.dx) && isfinite(h.dy);
}

// per-CTA shared histograms of dx and dy, added to the global ones once
__global__ void eta_hist_kernel(const pd_hit* __restrict__ hits, uint32_t n, uint32_t bins,
                                uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t sh[];  // [2][bins]
    for (uint32_t i = threadIdx.x; i < 2 * bins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const pd_hit h = hits[i];
        if (!single(h)) continue;
        uint32_t k;
        float phi;
        eta_bin(h.dx, bins, &k, &phi);
        atomicAdd(&sh[k], 1u);
        eta_bin(h.dy, bins, &k, &phi);
        atomicAdd(&sh[bins + k], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 2 * bins; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// counts below each bin, per axis (one thread per axis: bins are few)
__global__ void eta_cumulate_kernel(const uint32_t* __restrict__ hist, uint32_t bins,
                                    uint32_t* __restrict__ below) {
    const uint32_t a = threadIdx.x;
    if (a >= 2) return;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < bins; k++) {
        below[a * (bins + 1) + k] = acc;
        acc += hist[a * bins + k];
    }
    below[a * (bins + 1) + bins] = acc;
}

__device__ __forceinline__ float eta_map(float d, const uint32_t* __restrict__ h,
                                         const uint32_t* __restrict__ below, uint32_t bins) {
    const uint32_t n = below[bins];
    if (n == 0) return d;
    uint32_t k;
    float phi;
    eta_bin(d, bins, &k, &phi);
    const float num = __fadd_rn((float)below[k], __fmul_rn(phi, (float)h[k]));
    return __fsub_rn(__fdiv_rn(num, (float)n), 0.5f);
}

__global__ void eta_apply_kernel(const pd_hit* __restrict__ in, uint32_t n, uint32_t bins,
                                 const uint32_t* __restrict__ hist,
                                 const uint32_t* __restrict__ below, pd_hit* __restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        pd_hit h = in[i];
        if (single(h)) {
            h.dx = eta_map(h.dx, hist, below, bins);
            h.dy = eta_map(h.dy, hist + bins, below + bins + 1, bins);
            h.flags |= PD_HIT_LINEARISED;
        }
        out[i] = h;
    }
}

int eta_grid(uint32_t n) {
    const uint32_t g = (n + 255) / 256;
    const uint32_t cap = 4u * (uint32_t)pd::device_sm_count();
    return (int)(g < cap ? (g ? g : 1) : cap);
}

}  // namespace

extern "C" {

int pd_eta_create(uint32_t bins, pd_eta** out) {
    if (!out || bins > PD_MAX_ETA_BINS || !(bins & 1))
        return pd::internal_fail(PD_EINVAL, "pd_eta_create: bins odd, in [1, PD_MAX_ETA_BINS]");
    *out = nullptr;
    pd_eta* e = new (std::nothrow) pd_eta();
    if (!e) return pd::internal_fail(PD_ENOMEM, "host allocation failed");
    e->bins = bins;
    if (cudaMalloc(&e->hist, 2 * bins * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&e->below, 2 * (bins + 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(e->hist, 0, 2 * bins * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(e->below, 0, 2 * (bins + 1) * sizeof(uint32_t)) != cudaSuccess) {
        cudaFree(e->hist);
        cudaFree(e->below);
        delete e;
        return pd::internal_fail(PD_ENOMEM, "pd_eta_create: device allocation failed");
    }
    *out = e;
    return PD_OK;
}

int pd_eta_accumulate(pd_eta* e, const pd_hit* hits_dev, uint32_t n, void* stream) {
    if (!e || (n && !hits_dev)) return pd::internal_fail(PD_EINVAL, "pd_eta_accumulate: args");
    if (!n) return PD_OK;
    eta_hist_kernel<<<eta_grid(n), 256, 2 * e->bins * sizeof(uint32_t), (cudaStream_t)stream>>>(
        hits_dev, n, e->bins, e->hist);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? PD_OK
                              : pd::internal_fail(PD_ECUDA, cudaGetErrorString(err));
}

int pd_eta_finalize(pd_eta* e, void* stream) {
    if (!e) return pd::internal_fail(PD_EINVAL, "NULL eta");
    eta_cumulate_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(e->hist, e->bins, e->below);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? PD_OK
                              : pd::internal_fail(PD_ECUDA, cudaGetErrorString(err));
}

int pd_eta_apply(const pd_eta* e, const pd_hit* in_dev, uint32_t n, pd_hit* out_dev,
                 void* stream) {
    if (!e || (n && (!in_dev || !out_dev))) return pd::internal_fail(PD_EINVAL, "pd_eta_apply: args");
    if (!n) return PD_OK;
    eta_apply_kernel<<<eta_grid(n), 256, 0, (cudaStream_t)stream>>>(in_dev, n, e->bins, e->hist,
                                                                   e->below, out_dev);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? PD_OK
                              : pd::internal_fail(PD_ECUDA, cudaGetErrorString(err));
}

int pd_eta_get_histogram(const pd_eta* e, uint32_t* hist_host) {
    if (!e || !hist_host) return pd::internal_fail(PD_EINVAL, "NULL argument");
    const cudaError_t err = cudaMemcpy(hist_host, e->hist, 2 * e->bins * sizeof(uint32_t),
                                       cudaMemcpyDeviceToHost);
    return err == cudaSuccess ? PD_OK
                              : pd::internal_fail(PD_ECUDA, cudaGetErrorString(err));
}

int pd_eta_reset(pd_eta* e, void* stream) {
    if (!e) return pd::internal_fail(PD_EINVAL, "NULL eta");
    cudaError_t err =
        cudaMemsetAsync(e->hist, 0, 2 * e->bins * sizeof(uint32_t), (cudaStream_t)stream);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(e->below, 0, 2 * (e->bins + 1) * sizeof(uint32_t),
                              (cudaStream_t)stream);
    return err == cudaSuccess ? PD_OK
                              : pd::internal_fail(PD_ECUDA, cudaGetErrorString(err));
}

void pd_eta_destroy(pd_eta* e) {
    if (!e) return;
    cudaDeviceSynchronize();
    cudaFree(e->hist);
    cudaFree(e->below);
    delete e;
}

}  // extern "C"
