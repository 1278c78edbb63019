// pd_matched.cu — charge summing with the paper's matched filters.
//
// Section "Photon Charge Summing" (Figs. d, e) and section "Photon Subpixel
// Resolution" (Fig. f).  With T = (s > 0) the signal mask and s the zeroed
// signal, each feature f of the bank has four 4 x 5 filters F0, F1, F1dx,
// F1dy and a threshold F1Nmin:
//     Size_f = T * F1     Droplet_f = s * F1     Overflow_f = T * F0
//     Mx_f = s * F1dx     My_f = s * F1dy
//     Valid_f = (Overflow_f == 0) and (Size_f >= F1Nmin_f)
// and a pixel's energy is the sum of its valid droplets in feature order,
// its centroid the sum of Mx_f / Droplet_f (My_f / Droplet_f) over the valid
// features whose droplet is not 0.  A filter tap (i, j) applied at (r, c)
// meets (r + i - 1, c + j - 2), zero outside the module (TF's "SAME"
// alignment of a 4 x 5 kernel); each sum runs over the taps row-major from
// 0.0f with products rounded once.
//
// The bank is compiled on the host into lists of the nonzero taps.  Skipping
// a zero tap is exact: its term is +-0, and a sum that starts at +0.0f is
// never -0 (x + (-x) rounds to +0), so adding +-0 never changes it.  For the
// same reason a pixel whose 4 x 5 window holds no signal has every Size,
// Overflow and Droplet equal to 0, so its energy is 0 and it is skipped.
//
// matched_kernel: grid-stride over 16 x 64 tiles of (frame, module); the
// corrected signal of the tile and its halo (one row above, two below, two
// columns each side) goes to shared memory together with, per halo row and
// column, the 5-bit signal mask of the five columns around; four of those
// give a pixel's 20-bit window mask.  Pixels with a non-empty window
// evaluate the bank: Size is a popcount for features whose F1 taps are all
// 1, and Overflow == 0 a mask test for features whose F0 taps are all
// positive (a sum of positive terms is positive, and of ones is exact);
// other features, and the droplet and momenta of valid features, run over
// the tap lists.  Hits are compacted with a warp ballot and one atomic per
// warp.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kTY = 16, kTX = 64, kThreads = 256;
constexpr int kHY = kTY + 3, kHX = kTX + 4;

__device__ __forceinline__ uint32_t hist_bin(float v, float neg_lo_s, float inv_w,
                                             uint32_t bins) {
    const float t = __fmaf_rn(v, inv_w, neg_lo_s);
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)bins) return bins - 1;
    return (uint32_t)t;
}

template <bool STACKED, bool MG>
__global__ void __launch_bounds__(kThreads)
    matched_kernel(ChainParams p, const MatchedBank* __restrict__ bank,
                   const uint16_t* __restrict__ raw, uint32_t frame_base, CallOut out,
                   uint32_t tiles_y, uint32_t tiles_x, unsigned long long n_tiles,
                   MultiGain mg) {
    extern __shared__ uint32_t hsm[];  // [2][hist_bins]
    __shared__ float tile[kHY][kHX];
    __shared__ uint8_t row5[kHY][kTX];  // signal bits of columns c-2 .. c+2
    __shared__ uint32_t s_ucol[kHX], s_urow[kHY];  // unit offsets of halo columns / rows
    __shared__ MatchedBank sb;
    uint32_t* hpix = hsm;
    uint32_t* hhit = hsm + p.hist_bins;
    for (uint32_t b = threadIdx.x; b < 2 * p.hist_bins; b += kThreads) hsm[b] = 0;
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(bank);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sb);
        for (uint32_t k = threadIdx.x; k < sizeof(MatchedBank) / 4; k += kThreads) dst[k] = src[k];
    }
    __syncthreads();

    const int R = (int)p.rows, C = (int)p.cols;
    const int lane = threadIdx.x & 31;
    const uint32_t nf = sb.n_features;
    __shared__ uint32_t s_at[4];  // the tile's column, row, module and frame
    __shared__ uint32_t s_list[kTY * kTX];  // pixel j | window mask << 10
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
        const float* cmf = out.cm + (size_t)f * cm_per_frame(p) + (size_t)m * p.units_per_module;
        const float* cmr = out.cm + (size_t)f * cm_per_frame(p) + p.units_per_frame +
                           (size_t)m * p.rows;
        const float* cmc = out.cm + (size_t)f * cm_per_frame(p) + p.units_per_frame +
                           (size_t)p.n_modules * p.rows + (size_t)m * p.cols;

        // unit of each halo column and row (divisions per column and row, not
        // per pixel)
        for (int k = threadIdx.x; k < kHX + kHY; k += kThreads) {
            if (k < kHX) {
                const int c = c0 + k - 2;
                s_ucol[k] = c >= 0 && c < C ? (uint32_t)c / p.unit_cols : 0u;
            } else {
                const int r = r0 + (k - kHX) - 1;
                s_urow[k - kHX] = r >= 0 && r < R ? ((uint32_t)r / p.unit_rows) * p.units_per_row : 0u;
            }
        }
        __syncthreads();
        // 1. zeroed signal of the tile and its halo
        for (int j = threadIdx.x; j < kHY * kHX; j += kThreads) {
            const int hr = j / kHX, hc = j % kHX;
            const int r = r0 + hr - 1, c = c0 + hc - 2;
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
                if (hr >= 1 && hr <= kTY && hc >= 2 && hc < kTX + 2) {
                    atomicAdd(&hpix[hist_bin(e, p.hist_neg_lo_s, p.hist_inv_w, p.hist_bins)], 1u);
                    if (out.corrected)
                        out.corrected[(size_t)f * p.frame_px + mod_base + off] = e;
                }
            }
            tile[hr][hc] = s;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < kHY * kTX; j += kThreads) {
            const int hr = j / kTX, ic = j % kTX;
            const float* row = &tile[hr][ic];
            row5[hr][ic] = (uint8_t)((row[0] > 0.0f) | (row[1] > 0.0f) << 1 |
                                     (row[2] > 0.0f) << 2 | (row[3] > 0.0f) << 3 |
                                     (row[4] > 0.0f) << 4);
        }
        __syncthreads();

        // 2. pixels whose window holds signal into a list (warp-aggregated),
        //    so that the bank runs with every lane busy
        for (int base = 0; base < kTY * kTX; base += kThreads) {
            const int j = base + threadIdx.x;
            const int ir = j / kTX, ic = j % kTX;
            const uint32_t win = (uint32_t)row5[ir][ic] | (uint32_t)row5[ir + 1][ic] << 5 |
                                 (uint32_t)row5[ir + 2][ic] << 10 |
                                 (uint32_t)row5[ir + 3][ic] << 15;
            const bool cand = r0 + ir < R && c0 + ic < C && win;
            const uint32_t bal = __ballot_sync(0xffffffffu, cand);
            if (bal) {
                const int lead = __ffs(bal) - 1;
                uint32_t at0 = 0;
                if (lane == lead) at0 = atomicAdd(&s_nc, (uint32_t)__popc(bal));
                at0 = __shfl_sync(0xffffffffu, at0, lead);
                if (cand) s_list[at0 + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)j | win << 10;
            }
        }
        __syncthreads();
        const uint32_t n_cand = s_nc;

        // 3. the bank at the listed pixels
        for (uint32_t base = 0; base < n_cand; base += kThreads) {
            const uint32_t k = base + threadIdx.x;
            bool emit = false;
            pd_hit h;
            uint32_t n = 0, pix = 0;
            const uint32_t e_k = k < n_cand ? s_list[k] : 0u;
            const int j = (int)(e_k & 1023u);
            const uint32_t win = e_k >> 10;
            const int ir = j / kTX, ic = j % kTX;
            const int r = r0 + ir, c = c0 + ic;
            if (k < n_cand) {
                // window tap (i, j) is tile[ir + i][ic + j]
                const float* w = &tile[ir][ic];
                float E = 0.0f, dx = 0.0f, dy = 0.0f;
                uint32_t npix = 0;
                bool any = false;
                for (uint32_t ft = 0; ft < nf; ft++) {
                    bool clear;
                    if (sb.f0_pos[ft]) {
                        clear = (win & sb.m0[ft]) == 0;
                    } else {
                        float over = 0.0f;
                        for (uint32_t k = sb.off0[ft]; k < sb.off0[ft + 1]; k++)
                            if (w[sb.t0[k].at] > 0.0f) over = __fadd_rn(over, sb.t0[k].v);
                        clear = over == 0.0f;
                    }
                    if (!clear) continue;
                    float size;
                    if (sb.f1_unit[ft]) {
                        size = (float)__popc(win & sb.m1[ft]);
                    } else {
                        size = 0.0f;
                        for (uint32_t k = sb.off1[ft]; k < sb.off1[ft + 1]; k++)
                            if (w[sb.t1[k].at] > 0.0f) size = __fadd_rn(size, sb.t1[k].v);
                    }
                    if (!(size >= sb.nmin[ft])) continue;
                    float drop = 0.0f, mx = 0.0f, my = 0.0f;
                    uint32_t under = 0;
                    for (uint32_t k = sb.off1[ft]; k < sb.off1[ft + 1]; k++) {
                        const float sv = w[sb.t1[k].at];
                        drop = __fadd_rn(drop, __fmul_rn(sv, sb.t1[k].v));
                        under += sv > 0.0f;
                    }
                    for (uint32_t k = sb.offx[ft]; k < sb.offx[ft + 1]; k++)
                        mx = __fadd_rn(mx, __fmul_rn(w[sb.tx[k].at], sb.tx[k].v));
                    for (uint32_t k = sb.offy[ft]; k < sb.offy[ft + 1]; k++)
                        my = __fadd_rn(my, __fmul_rn(w[sb.ty[k].at], sb.ty[k].v));
                    if (!any) npix = under;
                    any = true;
                    E = __fadd_rn(E, drop);
                    if (drop != 0.0f) {
                        dx = __fadd_rn(dx, __fdiv_rn(mx, drop));
                        dy = __fadd_rn(dy, __fdiv_rn(my, drop));
                    }
                }
                if (any && E != 0.0f) {
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
                        if (r == 0 || c == 0 || r == R - 1 || c == C - 1) flags |= PD_HIT_EDGE;
                        pix = (uint32_t)mod_base + (uint32_t)r * p.cols + (uint32_t)c;
                        h.frame = frame_base + f;
                        h.pixel = pix;
                        h.energy_kev = E;
                        h.dx = dx;
                        h.dy = dy;
                        h.count = (uint8_t)n;
                        h.npix = (uint8_t)(npix > 255 ? 255 : npix);
                        h.flags = flags;
                        emit = true;
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
    for (uint32_t b = threadIdx.x; b < p.hist_bins; b += kThreads) {
        if (hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)hpix[b]);
        if (hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)hhit[b]);
    }
}

// Nonzero taps of one 4 x 5 filter, row-major, appended to list.
void compile_taps(const float (*flt)[5], MatchedTap* list, uint32_t* n) {
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 5; j++)
            if (flt[i][j] != 0.0f) {
                list[*n].at = (uint16_t)(i * kHX + j);
                list[*n].v = flt[i][j];
                (*n)++;
            }
}

}  // namespace

bool compile_bank(const pd_filter_bank& b, MatchedBank* out) {
    if (b.n_features < 1 || b.n_features > PD_MAX_FEATURES) return false;
    MatchedBank mb{};
    mb.n_features = b.n_features;
    uint32_t n1 = 0, n0 = 0, nx = 0, ny = 0;
    for (uint32_t f = 0; f < b.n_features; f++) {
        if (isnan(b.f1_nmin[f])) return false;
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 5; j++)
                if (!isfinite(b.f0[f][i][j]) || !isfinite(b.f1[f][i][j]) ||
                    !isfinite(b.f1_dx[f][i][j]) || !isfinite(b.f1_dy[f][i][j]))
                    return false;
        mb.nmin[f] = b.f1_nmin[f];
        mb.off1[f] = (uint16_t)n1;
        mb.off0[f] = (uint16_t)n0;
        mb.offx[f] = (uint16_t)nx;
        mb.offy[f] = (uint16_t)ny;
        compile_taps(b.f1[f], mb.t1, &n1);
        compile_taps(b.f0[f], mb.t0, &n0);
        mb.f1_unit[f] = mb.f0_pos[f] = 1;
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 5; j++) {
                if (b.f1[f][i][j] != 0.0f) {
                    mb.m1[f] |= 1u << (5 * i + j);
                    if (b.f1[f][i][j] != 1.0f) mb.f1_unit[f] = 0;
                }
                if (b.f0[f][i][j] != 0.0f) {
                    mb.m0[f] |= 1u << (5 * i + j);
                    if (!(b.f0[f][i][j] > 0.0f)) mb.f0_pos[f] = 0;
                }
            }
        compile_taps(b.f1_dx[f], mb.tx, &nx);
        compile_taps(b.f1_dy[f], mb.ty, &ny);
    }
    mb.off1[b.n_features] = (uint16_t)n1;
    mb.off0[b.n_features] = (uint16_t)n0;
    mb.offx[b.n_features] = (uint16_t)nx;
    mb.offy[b.n_features] = (uint16_t)ny;
    *out = mb;
    return true;
}

cudaError_t launch_matched(const ChainParams& p, const MatchedBank* bank_dev,
                           const uint16_t* raw, uint32_t n_frames, uint32_t frame_base,
                           const CallOut& out, cudaStream_t stream, const MultiGain* mg) {
    const uint32_t tiles_y = (p.rows + kTY - 1) / kTY;
    const uint32_t tiles_x = (p.cols + kTX - 1) / kTX;
    const unsigned long long n_tiles =
        (unsigned long long)n_frames * p.n_modules * tiles_y * tiles_x;
    if (n_tiles == 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)p.hist_bins * sizeof(uint32_t);
    static bool attr_set = false;
    if (!attr_set) {
        for (auto k : {matched_kernel<false, false>, matched_kernel<true, false>,
                       matched_kernel<false, true>}) {
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
        matched_kernel<false, true><<<(unsigned)grid, kThreads, smem, stream>>>(
            p, bank_dev, raw, frame_base, out, tiles_y, tiles_x, n_tiles, m);
    else if (cm_kind(p) == PD_CM_MEAN_STACKED)
        matched_kernel<true, false><<<(unsigned)grid, kThreads, smem, stream>>>(
            p, bank_dev, raw, frame_base, out, tiles_y, tiles_x, n_tiles, m);
    else
        matched_kernel<false, false><<<(unsigned)grid, kThreads, smem, stream>>>(
            p, bank_dev, raw, frame_base, out, tiles_y, tiles_x, n_tiles, m);
    return cudaGetLastError();
}

}  // namespace pd
