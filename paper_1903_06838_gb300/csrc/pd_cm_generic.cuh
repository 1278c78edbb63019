// pd_cm_generic.cuh — exact common mode of one unit by a 4-pass 8-bit radix
// select (paper section "Common Mode", Fig. c; lower median of d = raw -
// pedestal over d < cut, 0 when fewer than n_min pixels qualify).  Used for
// units of any size and shape; one CTA of any width handles one (frame,
// unit).  Keys are kept in shared memory when the unit fits, else recomputed
// from global memory on every pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_internal.cuh"

namespace pd {
namespace generic_cm {

constexpr uint32_t kSentinel = 0xFFFFFFFFu;  // "not in the common-mode set"

// Unsigned order of the keys == ascending IEEE order, with -0 below +0.
__device__ __forceinline__ uint32_t order_key(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

struct Shared {
    uint32_t hist[256];
    uint32_t warp_cnt[32];
    uint32_t s_prefix, s_rank;
};

// Common mode of unit `item` (= frame * units_per_frame + unit) into
// cm_out[item].  keys: unit_px words of shared memory when KEYS_IN_SMEM.
// MG: auto-ranging words (only stage-0 pixels enter the set; mg describes
// the stages).
template <bool KEYS_IN_SMEM, bool MG = false>
__device__ void unit(const ChainParams& p, const uint16_t* __restrict__ raw,
                     float* __restrict__ cm_out, uint32_t item, uint32_t* keys, Shared& sh,
                     const MultiGain& mg = MultiGain{}) {
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t f = item / p.units_per_frame;
    const uint32_t u = item % p.units_per_frame;
    if (cm_kind(p) == PD_CM_NONE) {
        if (tid == 0) cm_out[item] = 0.0f;
        return;
    }
    const uint32_t m = u / p.units_per_module;
    const uint32_t um = u % p.units_per_module;
    const uint32_t r0 = (um / p.units_per_row) * p.unit_rows;
    const uint32_t c0 = (um % p.units_per_row) * p.unit_cols;
    const size_t mod_base = (size_t)m * p.module_px;
    const uint16_t* fr = raw + (size_t)f * p.frame_px + mod_base;
    const float* pm = p.ped + mod_base;
    const float* gm = p.inv_gain + mod_base;
    const bool ag = cm_after_gain(p);

    auto key_at = [&](uint32_t i) -> uint32_t {
        const uint32_t off = (r0 + i / p.unit_cols) * p.cols + c0 + i % p.unit_cols;
        uint32_t w = fr[off];
        if (MG) {
            if ((w >> mg.shift) != 0) return kSentinel;
            w &= mg.vmask;
        }
        const float v =
            cm_input(ag, __fsub_rn(__uint2float_rn(w), pm[off]), ag ? gm[off] : 1.0f);
        return v < p.cm_cut ? order_key(v) : kSentinel;
    };

    uint32_t cnt = 0;
    for (uint32_t i = tid; i < p.unit_px; i += nthr) {
        const uint32_t k = key_at(i);
        if (KEYS_IN_SMEM) keys[i] = k;
        cnt += (k != kSentinel);
    }
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (nthr + 31) >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) sh.warp_cnt[warp] = cnt;
    __syncthreads();
    uint32_t n = 0;
    for (int w = 0; w < nwarps; w++) n += sh.warp_cnt[w];
    if (n == 0 || n < p.cm_min_count) {
        if (tid == 0) cm_out[item] = 0.0f;
        return;
    }
    if (tid == 0) {
        sh.s_prefix = 0;
        sh.s_rank = (n - 1) / 2;
    }
    // Radix select, most significant byte first.
    for (int pass = 0; pass < 4; pass++) {
        const int shift = 24 - 8 * pass;
        for (uint32_t b = tid; b < 256; b += nthr) sh.hist[b] = 0;
        __syncthreads();
        const uint32_t prefix = sh.s_prefix;
        for (uint32_t i = tid; i < p.unit_px; i += nthr) {
            const uint32_t k = KEYS_IN_SMEM ? keys[i] : key_at(i);
            if (k == kSentinel) continue;
            if (pass > 0 && (k >> (shift + 8)) != prefix) continue;
            atomicAdd(&sh.hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            // lane l owns bins 8l..8l+7
            uint32_t loc[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                loc[j] = sh.hist[lane * 8 + j];
                sum += loc[j];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t excl = incl - sum;
            const uint32_t rank = sh.s_rank;
            if (excl <= rank && rank < incl) {
                uint32_t below = excl;
                int digit = lane * 8;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    if (below + loc[j] > rank) {
                        digit = lane * 8 + j;
                        break;
                    }
                    below += loc[j];
                }
                sh.s_prefix = (prefix << 8) | (uint32_t)digit;
                sh.s_rank = rank - below;
            }
        }
        __syncthreads();
    }
    if (tid == 0) cm_out[item] = key_value(sh.s_prefix);
}

}  // namespace generic_cm
}  // namespace pd
