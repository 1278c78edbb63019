// pd_fast.cuh — configuration and launchers of the throughput kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pd_internal.cuh"

namespace pd {

constexpr uint32_t kCmBins = 4096;     // common-mode bins of 1/8 ADU (512 ADU)
constexpr uint32_t kCandCap = 2048;    // candidates of the winning bin
constexpr uint32_t kCmBigMinPx = 4096; // smaller units use the generic kernel (the
                                       // code buffer must hold kCandCap words)
constexpr size_t kCmBigMaxSmem = 112 * 1024;
constexpr uint32_t kBandThreads = 512;
constexpr uint32_t kSeedCap = 4096;    // seed candidates per band tile

struct CmBigConfig {
    float magic_w;  // 1.5*2^23 - 8*(cut - 512)
    float w_lo;     // cut - 512: lower edge of bin 0
    uint32_t vec;   // pixels per load (2 or 1)
    uint32_t tx, ty;
    bool ok;
};

struct BandConfig {
    uint32_t vec;     // pixels per chunk (4 or 1)
    uint32_t tx, ty;  // chunk columns x row lanes
    uint32_t pitch;   // floats per s-tile row
    uint32_t rb;      // rows per band
    uint32_t n_bands;
    bool ok;
};

// One item of a batched launch (device-side table entry).
struct BatchItem {
    ChainParams p;
    CmBigConfig cm_cfg;
    BandConfig band_cfg;
    uint32_t cm_kind;   // 0/1: large-unit kernel (2 or 1 pixels per load),
                        // 2/3: generic radix select (keys in shared / global),
                        // 4: one warp per small unit, 16 units per task
    float rows_magic;   // cm_rows_magic(p) for kind 4
    uint32_t band_vec;  // 4 or 1
    const uint16_t* raw;
    uint32_t n_frames, frame_base;
    CallOut out;                        // out.cm: this item's common mode
    unsigned long long cm_first;        // first common-mode task of the item
    unsigned long long st_first;        // first stencil tile of the item
    unsigned long long st_tiles;        // stencil tiles of the item
};

// Common mode of every item in one launch, then every stencil tile in one
// launch (both persistent), on `stream`.  all_kinds false: every item's
// common-mode kind is 0 or 4; vec: the band width all items share (4 or 1),
// or 0.
cudaError_t launch_batch(const BatchItem* items_dev, uint32_t n_items,
                         unsigned long long cm_tasks, size_t cm_smem, size_t band_smem,
                         cudaStream_t stream, bool all_kinds = true, int vec = 0);

CmBigConfig make_cm_big_config(const ChainParams& p);
bool cm_big_supported(const ChainParams& p, const CmBigConfig& cfg);
size_t cm_big_smem_bytes(const ChainParams& p);
// stage_mask: 0 for single-gain words; for auto-ranging words the stage bits
// (~value mask), whose pixels are not in stage 0 and stay out of the set.
cudaError_t launch_cm_big(const ChainParams& p, const CmBigConfig& cfg, const uint16_t* raw,
                          uint32_t n_frames, float* cm, cudaStream_t stream,
                          uint32_t stage_mask = 0);

// Units of at most 512 pixels (one warp each), cut an integer in (-1e6, 1e6).
float cm_rows_magic(const ChainParams& p);
bool cm_rows_supported(const ChainParams& p);
cudaError_t launch_cm_rows(const ChainParams& p, const uint16_t* raw, uint32_t n_frames,
                           float* cm, cudaStream_t stream);

BandConfig make_band_config(const ChainParams& p);
size_t band_smem_bytes(const ChainParams& p, uint32_t rb, uint32_t pitch);
// mg: auto-ranging words (four-pixel chunks and the median or no common
// mode only), or NULL.
cudaError_t launch_stencil_band(const ChainParams& p, const BandConfig& bc, const uint16_t* raw,
                                uint32_t n_frames, uint32_t frame_base, const CallOut& out,
                                cudaStream_t stream, const MultiGain* mg = nullptr);

// Whole chain in one persistent kernel per (frame, module) for modules whose
// common-mode units are full-height column banks (at most kFusedMaxUnits per
// module), or with common mode off; columns a multiple of 4.
constexpr uint32_t kFusedCmBins = 3584;  // bins of 1/8 ADU: window [cut - 448, cut)
constexpr uint32_t kFusedMaxUnits = 2;
#ifndef PD_FUSED_MAX_TY
#define PD_FUSED_MAX_TY 3
#endif
constexpr uint32_t kFusedMaxTy = PD_FUSED_MAX_TY;  // row lanes per CTA (registers: 2 CTAs / SM)

struct FusedConfig {
    float magic_w;                  // 1.5*2^23 - 8*(cut - 448)
    float w_lo;                     // cut - 448: lower edge of bin 0
    uint32_t tx, ty;                // chunk columns (cols / 4) x row lanes
    uint32_t pitch;                 // floats per ring row (cols + 8)
    uint32_t region_a_words;        // codes, then ring + seed lists
    uint32_t region_b_words;        // histograms, then candidates
    uint32_t smem_bytes;
    bool ok;
};

FusedConfig make_fused_config(const ChainParams& p);
cudaError_t launch_fused(const ChainParams& p, const FusedConfig& fc, const uint16_t* raw,
                         uint32_t n_frames, uint32_t frame_base, const CallOut& out,
                         cudaStream_t stream);

}  // namespace pd
