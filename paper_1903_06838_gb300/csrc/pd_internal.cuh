// pd_internal.cuh — device-side parameter block and kernel launchers shared
// by the translation units of libpd (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pd.h"

namespace pd {

// Everything a kernel needs to know about one detector context.  Passed by
// value as a kernel parameter (and stored in device memory for the batched
// launch), so it holds only plain values and device pointers.
struct ChainParams {
    // geometry
    uint32_t n_modules, rows, cols;
    uint32_t unit_rows, unit_cols;
    uint32_t units_per_row;     // cols / unit_cols
    uint32_t units_per_module;  // (rows / unit_rows) * units_per_row
    uint32_t unit_px;           // unit_rows * unit_cols
    uint32_t module_px;         // rows * cols
    uint32_t frame_px;          // n_modules * module_px
    uint32_t units_per_frame;
    uint32_t cm_mode;
    uint32_t cm_min_count;      // resolved n_min
    // thresholds
    float cm_cut, zero_thr, seed_thr, photon_kev;
    float hist_inv_w, hist_neg_lo_s;  // bin(v) = floor(fma(v, inv_w, neg_lo_s))
    uint32_t hist_bins;
    // device state owned by the context
    const float* ped;           // [frame_px]
    const float* nped;          // [frame_px] -pedestal (d = raw + nped)
    const float* inv_gain;      // [frame_px]
    uint32_t* count_map;        // [frame_px]
    unsigned long long* hist_pix;  // [hist_bins]
    unsigned long long* hist_hit;  // [hist_bins]
};

// Auto-ranging multi-gain data: each raw word holds its gain stage in the
// bits from `shift` up, the ADC value below; one pedestal and inverse-gain map
// per stage.  Passed beside ChainParams to the kernels that support it.
struct MultiGain {
    uint32_t n_gains, shift, vmask;
    const float* ped;       // [n_gains][frame_px]
    const float* inv_gain;  // [n_gains][frame_px]
};

// Energy of a multi-gain pixel (frame-relative index px) whose unit's common
// mode is cm: stage 0 subtracts the common mode, other stages do not, and a
// stage beyond the maps is a bad pixel with energy 0.
__device__ __forceinline__ float mg_energy(const MultiGain& mg, uint32_t frame_px, uint16_t w,
                                           size_t px, float cm) {
    const uint32_t st = (uint32_t)w >> mg.shift;
    if (st >= mg.n_gains) return 0.0f;
    const size_t at = (size_t)st * frame_px + px;
    const float d = __fsub_rn(__uint2float_rn((uint32_t)w & mg.vmask), mg.ped[at]);
    return __fmul_rn(st == 0 ? __fsub_rn(d, cm) : d, mg.inv_gain[at]);
}

// ChainParams.cm_mode holds the estimator (PD_CM_*) in its low byte and the
// paper's order (gain before common mode) as flag kCmAfterGain.
constexpr uint32_t kCmAfterGain = 0x100u;
__host__ __device__ inline uint32_t cm_kind(const ChainParams& p) { return p.cm_mode & 0xFFu; }
__host__ __device__ inline bool cm_after_gain(const ChainParams& p) {
    return (p.cm_mode & kCmAfterGain) != 0;
}

// The value a pixel brings to the common mode: d = raw - pedestal, or in
// the paper's order d * inv_gain (NaN, which no cut selects, for masked
// pixels).
__device__ __forceinline__ float cm_input(bool after_gain, float d, float inv_gain) {
    if (!after_gain) return d;
    return inv_gain != 0.0f ? __fmul_rn(d, inv_gain) : __int_as_float(0x7fc00000);
}

// Energy of a single-gain pixel from d, its unit's common mode and (stacked)
// the row and column terms, in the context's order.
template <bool STACKED>
__device__ __forceinline__ float energy(bool after_gain, float d, float inv_gain, float cm,
                                        float cmr, float cmc) {
    if (after_gain) {
        if (inv_gain == 0.0f) return 0.0f;
        float e = __fsub_rn(__fmul_rn(d, inv_gain), cm);
        if (STACKED) e = __fsub_rn(__fsub_rn(e, cmr), cmc);
        return e;
    }
    float c = __fsub_rn(d, cm);
    if (STACKED) c = __fsub_rn(__fsub_rn(c, cmr), cmc);
    return __fmul_rn(c, inv_gain);
}

// Common-mode values per frame: one per unit, then for the stacked mean one
// per module row and one per module column.
__host__ __device__ inline uint32_t cm_per_frame(const ChainParams& p) {
    return p.units_per_frame +
           (cm_kind(p) == PD_CM_MEAN_STACKED ? p.n_modules * (p.rows + p.cols) : 0u);
}

// A matched-filter bank compiled to lists of nonzero taps (pd_matched.cu).
// (i, j) is the tap's place in the 4 x 5 filter and `at` its offset in a
// kernel's shared tile, i * pitch + j (set for the tile kernel's pitch of 68;
// the band kernel rewrites it in its shared copy of the bank).
struct MatchedTap {
    uint8_t i, j;
    uint16_t at;
    float v;
};
struct MatchedBank {
    uint32_t n_features;
    float nmin[PD_MAX_FEATURES];
    // 20-bit masks of the nonzero F1 and F0 taps (bit 5 i + j), and whether
    // every nonzero F1 tap is 1 (Size = popcount) and every nonzero F0 tap
    // is positive (Overflow == 0 iff no signal under F0)
    uint32_t m1[PD_MAX_FEATURES], m0[PD_MAX_FEATURES];
    uint32_t f1_unit[PD_MAX_FEATURES], f0_pos[PD_MAX_FEATURES];
    uint16_t off1[PD_MAX_FEATURES + 1], off0[PD_MAX_FEATURES + 1];
    uint16_t offx[PD_MAX_FEATURES + 1], offy[PD_MAX_FEATURES + 1];
    MatchedTap t1[PD_MAX_FEATURES * 20], t0[PD_MAX_FEATURES * 20];
    MatchedTap tx[PD_MAX_FEATURES * 20], ty[PD_MAX_FEATURES * 20];
    // every feature binary (f1_unit and f0_pos): the valid features of a
    // pixel depend on its window mask alone, and vtab (device, 2^20 bytes,
    // or null) holds them for every mask
    uint32_t all_binary;
    const uint8_t* vtab;
};

// Per-call outputs (device pointers).
struct CallOut {
    pd_hit* hits;
    uint32_t hit_capacity;
    uint32_t* n_hits;
    float* corrected;  // may be null
    float* cm;         // [n_frames][cm_per_frame]; never null here
};

// Launchers (pd_chain.cu).  All are asynchronous on `stream` and return the
// CUDA launch status.
// mg: NULL for single-gain data.
cudaError_t launch_cm_select(const ChainParams& p, const uint16_t* raw,
                             uint32_t n_frames, float* cm, cudaStream_t stream,
                             const MultiGain* mg = nullptr);
cudaError_t launch_stencil(const ChainParams& p, const uint16_t* raw,
                           uint32_t n_frames, uint32_t frame_base,
                           const CallOut& out, cudaStream_t stream,
                           const MultiGain* mg = nullptr);
size_t cm_select_smem_bytes(const ChainParams& p);
// Matched-filter stencil (pd_matched.cu); compile_bank validates.
bool compile_bank(const pd_filter_bank& bank, MatchedBank* out);
// The valid-feature table of a bank whose features are all binary: 2^20
// bytes at vtab (synchronous).
cudaError_t build_vtab(const MatchedBank* bank_dev, uint8_t* vtab);
cudaError_t launch_matched(const ChainParams& p, const MatchedBank* bank_dev,
                           const uint16_t* raw, uint32_t n_frames, uint32_t frame_base,
                           const CallOut& out, cudaStream_t stream,
                           const MultiGain* mg = nullptr);
// The paper's mean estimator, one stage or three stacked (pd_cm_mean.cu).
cudaError_t launch_cm_mean(const ChainParams& p, const uint16_t* raw, uint32_t n_frames,
                           float* cm, cudaStream_t stream);

int device_sm_count();

// 5x5 patches of e / photon_kev around hits (pd_net.cu).
cudaError_t launch_gather(const ChainParams& p, const uint16_t* raw, uint32_t frame_base,
                          const float* cm, const pd_hit* hits, uint32_t n, float* patches,
                          cudaStream_t s, const MultiGain* mg = nullptr);

// Helpers of pd_process_noalloc (pd_api.cu).  None of them allocates.
int internal_fail(int code, const char* why);
int internal_check_process_args(const pd_ctx* ctx, const uint16_t* frames, uint32_t n_frames,
                                const pd_outputs* out, const char** why);
uint32_t internal_cm_per_frame(const pd_ctx* ctx);
int internal_ctx_device(const pd_ctx* ctx);
// false when the context runs the one-kernel chain (common mode on chip)
bool internal_uses_cm_scratch(const pd_ctx* ctx);
// pd_create: resolve the no-allocation scratch on device `dev` (current)
void noalloc_prepare(int dev);
// The chain on `stream` only (no second stream), with caller-provided
// common-mode storage of n_frames * cm_per_frame floats.
int internal_run_sequential(pd_ctx* ctx, const uint16_t* frames, uint32_t n_frames,
                            uint32_t frame_base, const pd_outputs* out, float* cm,
                            cudaStream_t stream);

}  // namespace pd
