// pd_chain.cu — the per-frame correction chain as two kernels:
//
//   cm_select_kernel  common mode of one unit (paper section "Common Mode",
//                     Fig. c): exact lower median of d = raw - pedestal over
//                     the unit's pixels with d < cut, found by a 4-pass
//                     8-bit radix select (pd_cm_generic.cuh).
//   stencil_kernel    dark, common mode (per unit; for the stacked mean also
//                     per module row and column) and gain correction (Fig. b), noise
//                     zeroing, 3x3 local maximum, charge sum, photon count
//                     (Fig. e), centre-of-mass offset (Fig. f), warp-ballot
//                     hit compaction and the summaries ("Summarization").
//
// Every floating-point operation is written as an explicit round-to-nearest
// intrinsic in the order the chain defines, and the file is compiled with
// --fmad=false, so results are reproducible bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_cm_generic.cuh"
#include "pd_dev.cuh"
#include "pd_internal.cuh"

namespace pd {

namespace {

__device__ __forceinline__ uint32_t hist_bin(float v, float neg_lo_s, float inv_w,
                                             uint32_t bins) {
    const float t = __fmaf_rn(v, inv_w, neg_lo_s);
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)bins) return bins - 1;
    return (uint32_t)t;  // truncation == floor for t >= 0
}

// ---------------------------------------------------------------------------
// Common mode: one CTA per (frame, unit).
constexpr int kCmThreads = 256;

template <bool KEYS_IN_SMEM, bool MG>
__global__ void __launch_bounds__(kCmThreads)
    cm_select_kernel(ChainParams p, const uint16_t* __restrict__ raw,
                     float* __restrict__ cm_out, MultiGain mg) {
    extern __shared__ uint32_t keys[];
    __shared__ generic_cm::Shared sh;
    generic_cm::unit<KEYS_IN_SMEM, MG>(p, raw, cm_out, blockIdx.x, keys, sh, mg);
}

// ---------------------------------------------------------------------------
// Stencil: grid-stride over TY x TX tiles of (frame, module).
constexpr int kTY = 16, kTX = 64, kStThreads = 256;
constexpr int kHY = kTY + 2, kHX = kTX + 2;

template <bool STACKED, bool MG>
__global__ void __launch_bounds__(kStThreads)
    stencil_kernel(ChainParams p, const uint16_t* __restrict__ raw,
                   uint32_t frame_base, CallOut out, uint32_t tiles_y,
                   uint32_t tiles_x, unsigned long long n_tiles, MultiGain mg) {
    extern __shared__ uint32_t hsm[];
    __shared__ float tile[kHY][kHX];
    __shared__ uint32_t s_ucol[kHX], s_urow[kHY];  // unit offsets of halo columns / rows
    uint32_t* hpix = hsm;
    uint32_t* hhit = hsm + p.hist_bins;
    for (uint32_t b = threadIdx.x; b < 2 * p.hist_bins; b += kStThreads) hsm[b] = 0;
    __syncthreads();

    const int R = (int)p.rows, C = (int)p.cols;
    const int lane = threadIdx.x & 31;
    __shared__ uint32_t s_at[4];  // the tile's column, row, module and frame
    __shared__ uint16_t s_list[kTY * kTX];  // the tile's seed candidates
    __shared__ uint32_t s_nc;
    for (unsigned long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        // one thread splits the tile index (64-bit divisions are long
        // instruction sequences; every thread doing them cost more than
        // the tile's pixels)
        if (threadIdx.x == 0) {
            unsigned long long q = t;
            s_at[0] = (uint32_t)(q % tiles_x);
            q /= tiles_x;
            s_at[1] = (uint32_t)(q % tiles_y);
            q /= tiles_y;
            s_at[2] = (uint32_t)(q % p.n_modules);
            s_at[3] = (uint32_t)(q / p.n_modules);
            s_nc = 0;
        }
        __syncthreads();
        const int tx = (int)s_at[0], ty = (int)s_at[1];
        const uint32_t m = s_at[2], f = s_at[3];
        const int r0 = ty * kTY, c0 = tx * kTX;
        const size_t mod_base = (size_t)m * p.module_px;
        const uint16_t* fr = raw + (size_t)f * p.frame_px + mod_base;
        const float* cmf = out.cm + (size_t)f * cm_per_frame(p) +
                           (size_t)m * p.units_per_module;
        // stacked mean: module-row and module-column terms after the units'
        const float* cmr = out.cm + (size_t)f * cm_per_frame(p) + p.units_per_frame +
                           (size_t)m * p.rows;
        const float* cmc = out.cm + (size_t)f * cm_per_frame(p) + p.units_per_frame +
                           (size_t)p.n_modules * p.rows + (size_t)m * p.cols;

        // unit of each halo column and row (two divisions per column and row
        // of the tile rather than per pixel)
        for (int k = threadIdx.x; k < kHX + kHY; k += kStThreads) {
            if (k < kHX) {
                const int c = c0 + k - 1;
                s_ucol[k] = c >= 0 && c < C ? (uint32_t)c / p.unit_cols : 0u;
            } else {
                const int r = r0 + (k - kHX) - 1;
                s_urow[k - kHX] = r >= 0 && r < R ? ((uint32_t)r / p.unit_rows) * p.units_per_row : 0u;
            }
        }
        __syncthreads();
        // 1. corrected signal of the tile and its 1-pixel halo
        for (int j = threadIdx.x; j < kHY * kHX; j += kStThreads) {
            const int hr = j / kHX, hc = j % kHX;
            const int r = r0 + hr - 1, c = c0 + hc - 1;
            float s = 0.0f;
            if (r >= 0 && r < R && c >= 0 && c < C) {
                const uint32_t off = (uint32_t)r * p.cols + (uint32_t)c;
                const float cm = cmf[s_urow[hr] + s_ucol[hc]];
                float e;
                if (MG) {
                    e = mg_energy(mg, p.frame_px, fr[off], mod_base + off, cm);
                } else {
                    const float d = __fsub_rn(__uint2float_rn(fr[off]), p.ped[mod_base + off]);
                    e = energy<STACKED>(cm_after_gain(p), d, p.inv_gain[mod_base + off], cm,
                                        STACKED ? cmr[r] : 0.0f, STACKED ? cmc[c] : 0.0f);
                }
                s = e > p.zero_thr ? e : 0.0f;
                if (hr >= 1 && hr <= kTY && hc >= 1 && hc <= kTX) {
                    atomicAdd(&hpix[hist_bin(e, p.hist_neg_lo_s, p.hist_inv_w, p.hist_bins)], 1u);
                    if (out.corrected)
                        out.corrected[(size_t)f * p.frame_px + mod_base + off] = e;
                }
            }
            tile[hr][hc] = s;
        }
        __syncthreads();

        // 2. pixels above the seed threshold into a list (warp-aggregated), so
        //    that the seed tests below run with every lane busy
        for (int base = 0; base < kTY * kTX; base += kStThreads) {
            const int j = base + threadIdx.x;
            const int ir = j / kTX, ic = j % kTX;
            const bool cand = r0 + ir < R && c0 + ic < C && tile[ir + 1][ic + 1] > p.seed_thr;
            const uint32_t bal = __ballot_sync(0xffffffffu, cand);
            if (bal) {
                const int lead = __ffs(bal) - 1;
                uint32_t at0 = 0;
                if (lane == lead) at0 = atomicAdd(&s_nc, (uint32_t)__popc(bal));
                at0 = __shfl_sync(0xffffffffu, at0, lead);
                if (cand) s_list[at0 + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)j;
            }
        }
        __syncthreads();
        const uint32_t n_cand = s_nc;

        // 3. seeds, sums, count, centroid; warp-aggregated emission
        for (uint32_t base = 0; base < n_cand; base += kStThreads) {
            const uint32_t k = base + threadIdx.x;
            bool emit = false;
            pd_hit h;
            uint32_t n = 0, pix = 0;
            if (k < n_cand) {
                const int j = s_list[k];
                const int ir = j / kTX, ic = j % kTX;
                const int r = r0 + ir, c = c0 + ic;
                const float sp = tile[ir + 1][ic + 1];
                {
                    bool seed = true;
#pragma unroll
                    for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                        for (int dx = -1; dx <= 1; dx++) {
                            if (!dy && !dx) continue;
                            const float sq = tile[ir + 1 + dy][ic + 1 + dx];
                            const bool before = dy < 0 || (dy == 0 && dx < 0);
                            seed = seed && (before ? (sp > sq) : (sp >= sq));
                        }
                    if (seed) {
                        float E = 0.0f, Mx = 0.0f, My = 0.0f;
                        uint32_t npix = 0;
#pragma unroll
                        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                            for (int dx = -1; dx <= 1; dx++) {
                                const float sq = tile[ir + 1 + dy][ic + 1 + dx];
                                E = __fadd_rn(E, sq);
                                Mx = __fadd_rn(Mx, __fmul_rn(sq, (float)dx));
                                My = __fadd_rn(My, __fmul_rn(sq, (float)dy));
                                npix += sq > 0.0f;
                            }
                        atomicAdd(&hhit[hist_bin(E, p.hist_neg_lo_s, p.hist_inv_w, p.hist_bins)], 1u);
                        const float qr = rintf(__fdiv_rn(E, p.photon_kev));
                        uint16_t flags = 0;
                        if (!(qr >= 0.0f)) {
                            n = 0;
                        } else if (qr > 255.0f) {
                            n = 255;
                            flags |= PD_HIT_SATURATED;
                        } else {
                            n = (uint32_t)qr;
                        }
                        if (n >= 1) {
                            if (r == 0 || c == 0 || r == R - 1 || c == C - 1)
                                flags |= PD_HIT_EDGE;
                            pix = (uint32_t)mod_base + (uint32_t)r * p.cols + (uint32_t)c;
                            h.frame = frame_base + f;
                            h.pixel = pix;
                            h.energy_kev = E;
                            h.dx = moment_over_energy(Mx, E);
                            h.dy = moment_over_energy(My, E);
                            h.count = (uint8_t)n;
                            h.npix = (uint8_t)npix;
                            h.flags = flags;
                            emit = true;
                        }
                    }
                }
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, emit);
            if (mask) {
                uint32_t slot = 0;
                if (lane == __ffs(mask) - 1) slot = atomicAdd(out.n_hits, __popc(mask));
                slot = __shfl_sync(0xffffffffu, slot, __ffs(mask) - 1);
                if (emit) {
                    slot += __popc(mask & ((1u << lane) - 1u));
                    atomicAdd(&p.count_map[pix], n);
                    if (slot < out.hit_capacity) out.hits[slot] = h;
                }
            }
        }
        __syncthreads();
    }
    for (uint32_t b = threadIdx.x; b < p.hist_bins; b += kStThreads) {
        if (hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)hpix[b]);
        if (hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)hhit[b]);
    }
}

}  // namespace

size_t cm_select_smem_bytes(const ChainParams& p) {
    return (size_t)p.unit_px * sizeof(uint32_t);
}

static constexpr size_t kMaxDynSmem = 200 * 1024;

cudaError_t launch_cm_select(const ChainParams& p, const uint16_t* raw,
                             uint32_t n_frames, float* cm, cudaStream_t stream,
                             const MultiGain* mg) {
    const unsigned long long items = (unsigned long long)n_frames * p.units_per_frame;
    if (items == 0) return cudaSuccess;
    const size_t smem = cm_select_smem_bytes(p);
    const MultiGain m = mg ? *mg : MultiGain{};
    if (smem <= kMaxDynSmem) {
        static bool attr_set = false;
        if (!attr_set) {
            for (auto k : {cm_select_kernel<true, false>, cm_select_kernel<true, true>}) {
                cudaError_t e = cudaFuncSetAttribute(
                    k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
                if (e != cudaSuccess) return e;
            }
            attr_set = true;
        }
        if (mg)
            cm_select_kernel<true, true><<<(unsigned)items, kCmThreads, smem, stream>>>(p, raw, cm, m);
        else
            cm_select_kernel<true, false><<<(unsigned)items, kCmThreads, smem, stream>>>(p, raw, cm, m);
    } else if (mg) {
        cm_select_kernel<false, true><<<(unsigned)items, kCmThreads, 0, stream>>>(p, raw, cm, m);
    } else {
        cm_select_kernel<false, false><<<(unsigned)items, kCmThreads, 0, stream>>>(p, raw, cm, m);
    }
    return cudaGetLastError();
}

cudaError_t launch_stencil(const ChainParams& p, const uint16_t* raw,
                           uint32_t n_frames, uint32_t frame_base,
                           const CallOut& out, cudaStream_t stream, const MultiGain* mg) {
    const uint32_t tiles_y = (p.rows + kTY - 1) / kTY;
    const uint32_t tiles_x = (p.cols + kTX - 1) / kTX;
    const unsigned long long n_tiles =
        (unsigned long long)n_frames * p.n_modules * tiles_y * tiles_x;
    if (n_tiles == 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)p.hist_bins * sizeof(uint32_t);
    static bool attr_set = false;
    if (!attr_set) {
        for (auto k : {stencil_kernel<false, false>, stencil_kernel<true, false>,
                       stencil_kernel<false, true>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(2 * PD_MAX_HIST_BINS * sizeof(uint32_t)));
            if (e != cudaSuccess) return e;
        }
        attr_set = true;
    }
    unsigned long long grid = (unsigned long long)device_sm_count() * 4;
    if (grid > n_tiles) grid = n_tiles;
    const MultiGain m = mg ? *mg : MultiGain{};
    if (mg)
        stencil_kernel<false, true><<<(unsigned)grid, kStThreads, smem, stream>>>(
            p, raw, frame_base, out, tiles_y, tiles_x, n_tiles, m);
    else if (cm_kind(p) == PD_CM_MEAN_STACKED)
        stencil_kernel<true, false><<<(unsigned)grid, kStThreads, smem, stream>>>(
            p, raw, frame_base, out, tiles_y, tiles_x, n_tiles, m);
    else
        stencil_kernel<false, false><<<(unsigned)grid, kStThreads, smem, stream>>>(
            p, raw, frame_base, out, tiles_y, tiles_x, n_tiles, m);
    return cudaGetLastError();
}

}  // namespace pd
