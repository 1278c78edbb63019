// pd_lean.cuh — configuration and launchers of the lean kernel pair
// (pd_lean.cu): the integer-coded bank median and the stencil that keeps
// corrected energies in shared memory and tests only seed candidates.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pd_fast.cuh"
#include "pd_internal.cuh"

namespace pd {

// Integer bin codes of the common-mode histogram.  For pixel p and raw word
// x, the bin floor(8 (d - lo)) of d = x - ped_p equals 8 x + F_p with
// F_p = floor(-8 (ped_p + lo)) whenever d is exact in binary32 (which the
// context checks for every d inside the window [lo, cut)); outside the
// window both forms clamp to the same end.  Codes are kept biased by `bias`
// in 16-bit lanes, two pixels per 32-bit word:
//   code' = clamp(8 min(x, rcap) + K'_p, bias, bias + 4096),
//   K'_p = F_p + bias,
// and bias + 4096 is the spare bin (d >= cut).  The map holds K' in the
// layout of the kernel's shared-memory copy of each unit: the frames are
// read as the tensor [frame][period][16-byte group][8 words] (a period is
// t rows, t cols a multiple of 8 words), and a unit's rows of one phase
// (row mod t) are one box of bp periods x w8 groups, padded to ne_box
// groups.  Slots that hold other pixels carry bias + 4096, so they land in
// the spare bin.
struct CodeMap {
    const uint4* kmap;  // [units_per_frame][t][ne_box] groups of 8 lanes
    uint32_t w8;        // groups per box row
    uint32_t bias;      // code' - code
    uint32_t rcap;      // raw words are clamped to rcap before coding
    uint32_t t;         // rows per period
    uint32_t bp;        // periods per box
    uint32_t ne_box;    // groups per staged box (bp * w8 rounded up to 8)
    uint32_t ctas_per_sm;  // persistent CTAs per SM of a launch
    uint32_t wait_polls;   // polls of a copy's mbarrier before giving up (0: default)
};

// Host side: the map of a geometry and pedestal (out->kmap left null), or
// false when the integer codes are not exact, do not fit 16-bit lanes, or the
// boxes exceed the tensor copy's limits (the context then keeps the
// floating-point bank median).  lo = cut - 512 (the window of
// make_cm_big_config).
bool build_code_map(const ChainParams& p, const float* pedestal, std::vector<uint16_t>* kmap,
                    CodeMap* out);
size_t cm_bank_smem_bytes(const ChainParams& p, const CodeMap& cmap);
bool cm_bank_supported(const ChainParams& p, const CodeMap& cmap);
// err: context error word (bit 0: a bounded wait for the staged copies gave
// up).  raw: 16-byte aligned frames of frame_px % 8 == 0 words.
cudaError_t launch_cm_bank(const ChainParams& p, const CmBigConfig& cfg, const CodeMap& cmap,
                           const uint16_t* raw, uint32_t n_frames, float* cm, uint32_t* err,
                           cudaStream_t stream);

// Lean stencil over bands of full-width rows (four-pixel chunks).
struct LeanConfig {
    uint32_t tx, ty;     // chunk columns (cols / 4) x row lanes
    uint32_t rb;         // rows per band
    uint32_t n_bands;
    uint32_t pitch;      // floats per tile row: 4 zero columns, cols, 4 zero columns
    uint32_t colbank;    // 1: units span the module's full height
    uint32_t list_cap;   // seed candidates per tile
    uint32_t ctas_per_sm;  // persistent CTAs per SM of a launch (0: as shared memory allows)
    // staged raw (stage_t > 0): each tile's rows, halo rows included, come
    // to shared memory as one tensor copy of stage_bp periods of stage_t
    // rows (frames read as [frame][period][16-byte group][8 words], stage_g
    // groups per period); the next tile's copy is in flight while a tile's
    // seeds are tested
    uint32_t stage_t, stage_g, stage_bp;
    uint32_t wait_polls;  // polls of a staged copy or a tile's dependency (0: default)
    bool ok;
};

LeanConfig make_lean_config(const ChainParams& p, uint32_t rb = 0);
size_t lean_smem_bytes(const ChainParams& p, const LeanConfig& lc);
// raw: 16-byte aligned.  err: context error word (bit 1: a bounded wait
// for a staged copy gave up).
cudaError_t launch_stencil_lean(const ChainParams& p, const LeanConfig& lc, const uint16_t* raw,
                                uint32_t n_frames, uint32_t frame_base, const CallOut& out,
                                uint32_t* err, cudaStream_t stream);

// The lean pair as one persistent launch over a work queue (bank items of
// frames [sK, sK + K) then the stencil tiles of the K frames before them, K
// frames of raw staying in L2 between the two), for column-bank units and
// the unstaged stencil without corrected frames.  out.cm receives the common
// mode of all n_frames.  qsync: queue_sync_words(p, n_frames) words of
// device scratch (cleared by the launch).  err bits: 1 a staged copy's wait,
// 4 a tile's wait for its banks gave up.
size_t queue_smem_bytes(const ChainParams& p, const CodeMap& cmap, const LeanConfig& lc);
bool queue_supported(const ChainParams& p, const CodeMap& cmap, const LeanConfig& lc);
size_t queue_sync_words(const ChainParams& p, uint32_t n_frames);
cudaError_t launch_chain_queue(const ChainParams& p, const CmBigConfig& cfg, const CodeMap& cmap,
                               const LeanConfig& lc, const uint16_t* raw, uint32_t n_frames,
                               uint32_t frame_base, const CallOut& out, uint32_t* qsync,
                               uint32_t* err, cudaStream_t stream);

}  // namespace pd
