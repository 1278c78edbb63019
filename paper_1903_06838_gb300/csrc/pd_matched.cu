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
// the tap lists (a bank of binary features reads its valid features from the
// table described below).  Hits are compacted with a warp ballot and one
// atomic per warp.
//
// matched_band_kernel: the same per pixel on full-width bands of module rows
// (single gain, raw - pedestal before the common mode), with the band
// stencil's four-pixel vector loads and packed correction.  Each thread
// stores the signal bits of its four pixels as one nibble (a pixel's window
// mask is read from the nibbles of four rows), and a chunk with signal marks
// the pixels whose windows it lies in on a bitmap of the band, from which
// the candidate list is built.  The valid features of every candidate come
// first (for a bank of binary features, from a table indexed by the window
// mask); the sums then run over a second list of the candidates with a valid
// feature, so that they keep every lane busy.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "pd_dev.cuh"
#include "pd_fast.cuh"
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

// The bank at one pixel: w points at its window's tap (0, 0) in a shared
// tile (tap (i, j) at w[i * pitch + j], the pitch folded into the taps'
// offsets), win is its 20-bit signal mask.  valid_features gives the mask
// of the valid features; sum_features their energy E, centroid sums dx, dy
// and npix (the signal pixels under the first valid feature's F1), as
// described above.
__device__ __forceinline__ uint32_t valid_features(const MatchedBank& sb, const float* w,
                                                   uint32_t win) {
    if (sb.vtab) return sb.vtab[win];
    uint32_t valid = 0;
    for (uint32_t ft = 0; ft < sb.n_features; ft++) {
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
        if (size >= sb.nmin[ft]) valid |= 1u << ft;
    }
    return valid;
}

__device__ __forceinline__ void sum_features(const MatchedBank& sb, const float* w,
                                             uint32_t valid, float& E, float& dx, float& dy,
                                             uint32_t& npix) {
    E = dx = dy = 0.0f;
    npix = 0;
    bool any = false;
    while (valid) {
        const uint32_t ft = (uint32_t)(__ffs(valid) - 1);
        valid &= valid - 1;
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
}

// Count, flags and record of a pixel whose bank gave energy E (E != 0);
// returns whether it is a hit (count >= 1) and adds E to the hit histogram.
__device__ __forceinline__ bool make_hit(const ChainParams& p, uint32_t* hhit, float E, float dx,
                                         float dy, uint32_t npix, int r, int c, uint32_t frame,
                                         size_t mod_base, pd_hit& h, uint32_t& n, uint32_t& pix) {
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
    if (n < 1) return false;
    const int R = (int)p.rows, C = (int)p.cols;
    if (r == 0 || c == 0 || r == R - 1 || c == C - 1) flags |= PD_HIT_EDGE;
    pix = (uint32_t)mod_base + (uint32_t)r * p.cols + (uint32_t)c;
    h.frame = frame;
    h.pixel = pix;
    h.energy_kev = E;
    h.dx = dx;
    h.dy = dy;
    h.count = (uint8_t)n;
    h.npix = (uint8_t)(npix > 255 ? 255 : npix);
    h.flags = flags;
    return true;
}

// Warp-aggregated emission: one atomic on the hit counter per warp.  wm:
// the warp's lanes (all of them must call).
__device__ __forceinline__ void emit_hits(const ChainParams& p, const CallOut& out, bool emit,
                                          const pd_hit& h, uint32_t n, uint32_t pix, int lane,
                                          unsigned wm = 0xffffffffu) {
    const uint32_t mask = __ballot_sync(wm, emit);
    if (mask) {
        uint32_t slot = 0;
        if (lane == __ffs(mask) - 1) slot = atomicAdd(out.n_hits, __popc(mask));
        slot = __shfl_sync(wm, slot, __ffs(mask) - 1);
        if (emit) {
            slot += __popc(mask & ((1u << lane) - 1u));
            atomicAdd(&p.count_map[pix], n);
            if (slot < out.hit_capacity) out.hits[slot] = h;
        }
    }
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
                const uint32_t valid = valid_features(sb, &tile[ir][ic], win);
                if (valid) {
                    float E, dx, dy;
                    uint32_t npix;
                    sum_features(sb, &tile[ir][ic], valid, E, dx, dy, npix);
                    if (E != 0.0f)
                        emit = make_hit(p, hhit, E, dx, dy, npix, r, c, frame_base + f, mod_base,
                                        h, n, pix);
                }
            }
            emit_hits(p, out, emit, h, n, pix, lane);
        }
        __syncthreads();
    }
    for (uint32_t b = threadIdx.x; b < p.hist_bins; b += kThreads) {
        if (hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)hpix[b]);
        if (hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)hhit[b]);
    }
}

// Candidates per band tile (a larger count tests every own pixel).
constexpr uint32_t kMbCap = 3072;

// Shared memory of the band kernel for bands of rb rows: the s-tile of
// rb + 3 rows (one above, two below) at the given pitch, both histograms
// (plus a spare bin), the candidate list and the list of those with a valid
// feature, the negated common mode of every (tile row, unit column), the
// stacked row terms, the candidate bitmap of the own rows and the signal
// nibbles.
size_t band_smem(const ChainParams& p, uint32_t rb, uint32_t pitch) {
    const size_t nr = rb + 3;
    return 4 * (nr * pitch + 2 * (size_t)p.hist_bins + 4 + 2 * kMbCap + nr * p.units_per_row +
                nr + (size_t)(rb + 1) * ((pitch + 31) / 32)) +
           nr * (pitch / 4);
}

constexpr uint32_t kMaxTaps = PD_MAX_FEATURES * 20;

// Bands of rb rows of (frame, module): tile t is band t % n_bands of module
// (t / n_bands) % n_modules of frame t / (n_bands * n_modules).
template <bool STACKED>
__global__ void __launch_bounds__(kBandThreads, 2)
    matched_band_kernel(ChainParams p, const MatchedBank* __restrict__ bank,
                        const uint16_t* __restrict__ raw, uint32_t frame_base, CallOut out,
                        BandConfig bc, unsigned long long n_tiles) {
    extern __shared__ __align__(16) uint32_t msm[];
    __shared__ MatchedBank sb;
    __shared__ uint32_t s_nc, s_nv;
    const uint32_t P = bc.pitch, NQ = P / 4, NR = bc.rb + 3;
    float* stile = reinterpret_cast<float*>(msm);  // NR x P; real column c at 4 + c
    uint32_t* hpix = msm + NR * P;                 // hist_bins + spare
    uint32_t* hhit = hpix + p.hist_bins + 4;       // hist_bins
    uint32_t* list = hhit + p.hist_bins;           // kMbCap: row << 16 | column
    uint32_t* vlist = list + kMbCap;               // kMbCap: list index | valid << 24
    float* cmt = reinterpret_cast<float*>(vlist + kMbCap);  // NR x units_per_row
    float* crt = cmt + NR * p.units_per_row;                  // NR row terms
    // candidate bitmap: bit x of row rl (words of WPR per row, rows 1 ..
    // rows_here used) marks s-tile column x of own row rl as a pixel whose
    // window holds signal; zero between tiles
    const uint32_t WPR = (P + 31) / 32;
    uint32_t* cbits = reinterpret_cast<uint32_t*>(crt + NR);  // (rb + 1) x WPR
    // nibble q of a row: signal bits of s-tile columns 4q .. 4q + 3 (real
    // columns 4q - 4 .. 4q - 1); the first and last nibble stay 0
    uint8_t* nib = reinterpret_cast<uint8_t*>(cbits + (bc.rb + 1) * WPR);

    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31;
    const int R = (int)p.rows, C = (int)p.cols;
    const uint32_t TX = bc.tx, TY = bc.ty;
    const uint32_t tx = tid % TX, ty = tid / TX;
    const bool active = ty < TY;
    const int col = (int)(tx * 4);  // first column of this thread's chunk
    const uint32_t uca = (uint32_t)col / p.unit_cols;
    const uint32_t ucb = (uint32_t)(col + 3) / p.unit_cols;
    const int split = (int)(ucb * p.unit_cols) - col;  // pixels i >= split use ucb
    const int max_bits = (int)(kMagicBits + p.hist_bins - 1);
    const int trash_bits = (int)(kMagicBits + p.hist_bins);

    for (uint32_t i = tid; i < NR * P; i += nthr) stile[i] = 0.0f;
    for (uint32_t i = tid; i < NR * NQ; i += nthr) nib[i] = 0;
    for (uint32_t i = tid; i < (bc.rb + 1) * WPR; i += nthr) cbits[i] = 0;
    for (uint32_t i = tid; i < 2 * p.hist_bins + 4; i += nthr) hpix[i] = 0;
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(bank);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sb);
        for (uint32_t k = tid; k < sizeof(MatchedBank) / 4; k += nthr) dst[k] = src[k];
    }
    __syncthreads();
    // tap offsets at this pitch
    for (uint32_t k = tid; k < 4 * kMaxTaps; k += nthr) {
        MatchedTap* lst = k < kMaxTaps ? sb.t1 : k < 2 * kMaxTaps ? sb.t0
                                             : k < 3 * kMaxTaps ? sb.tx : sb.ty;
        MatchedTap& tp = lst[k % kMaxTaps];
        tp.at = (uint16_t)(tp.i * P + tp.j);
    }

    // negated common mode of entry i (tile row, unit column) of tile tt; each
    // thread holds its entry of the next tile in a register
    const uint32_t ncmt = NR * p.units_per_row;
    auto tile_cm = [&](unsigned long long tt, uint32_t i) -> float {
        const unsigned long long fm = tt / bc.n_bands;
        const int r = (int)(tt - fm * bc.n_bands) * (int)bc.rb - 1 + (int)(i / p.units_per_row);
        if (r < 0 || r >= R) return 0.0f;
        const size_t fbase = (size_t)fm * p.units_per_module +
                             (STACKED ? (size_t)(fm / p.n_modules) *
                                            (cm_per_frame(p) - p.units_per_frame)
                                      : 0);
        return -out.cm[fbase + ((uint32_t)r / p.unit_rows) * p.units_per_row +
                       i % p.units_per_row];
    };
    float cmv = 0.0f;
    if (blockIdx.x < n_tiles && tid < ncmt) cmv = tile_cm(blockIdx.x, tid);

    TileWalk walk(blockIdx.x, gridDim.x, bc.n_bands, p.n_modules);
    // the last thread asks L2 for the raw rows (the halo row above, two
    // below) of the next tile now and of the tile after next once a tile is
    // done, so that their loads find them there
    const unsigned long long step = gridDim.x;
    const bool prefetcher = tid == nthr - 1;
    if (prefetcher && blockIdx.x + step < n_tiles) {
        TileWalk nx = walk;
        nx.next();
        prefetch_tile_rows(raw, nx, bc.rb, p.rows, p.cols, p.frame_px, 2);
    }
    for (unsigned long long t = blockIdx.x; t < n_tiles; t += gridDim.x, walk.next()) {
        const int band = (int)walk.band;
        const uint32_t m = walk.m, f = walk.f;
        const int r0 = band * (int)bc.rb;
        const int rows_here = min((int)bc.rb, R - r0);
        const size_t mod_base = (size_t)m * p.module_px;
        const uint16_t* fr = raw + (size_t)f * p.frame_px + mod_base;
        const float* npm = p.nped + mod_base;
        const float* gm = p.inv_gain + mod_base;

        if (tid < ncmt) cmt[tid] = cmv;
        for (uint32_t i = tid + nthr; i < ncmt; i += nthr) cmt[i] = tile_cm(t, i);
        float ncc[4];
        if (STACKED) {
            const float* cmf = out.cm + (size_t)f * cm_per_frame(p) + p.units_per_frame;
            for (uint32_t i = tid; i < NR; i += nthr) {
                const int r = r0 - 1 + (int)i;
                crt[i] = r >= 0 && r < R ? -cmf[(size_t)m * p.rows + r] : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
                ncc[i] = active ? -cmf[(size_t)p.n_modules * p.rows + (size_t)m * p.cols + col + i]
                                : 0.0f;
        }
        if (tid == 0) s_nc = s_nv = 0;
        __syncthreads();

        // 1. zeroed signal and its nibbles of rows r0-1 .. r0+rows_here+1;
        //    halo rows are not histogrammed (their bins go to the spare bin)
        if (active) {
            const int nrows = rows_here + 3;
            constexpr int U = 1;
            for (int rl0 = (int)ty; rl0 < nrows; rl0 += U * (int)TY) {
                uint2 rr[U];
                float4 pp[U], gg[U];
                bool in[U];
#pragma unroll
                for (int j = 0; j < U; j++) {
                    const int rl = rl0 + j * (int)TY;
                    const int r = r0 - 1 + rl;
                    in[j] = rl < nrows && r >= 0 && r < R;
                    if (in[j]) {
                        const uint32_t off = (uint32_t)r * p.cols + (uint32_t)col;
                        rr[j] = *reinterpret_cast<const uint2*>(fr + off);
                        pp[j] = *reinterpret_cast<const float4*>(npm + off);
                        gg[j] = *reinterpret_cast<const float4*>(gm + off);
                    }
                }
#pragma unroll
                for (int j = 0; j < U; j++) {
                    const int rl = rl0 + j * (int)TY;
                    if (rl >= nrows) continue;
                    float* srow = stile + rl * P + 4 + col;
                    uint8_t* nq = nib + rl * NQ + tx + 1;
                    if (!in[j]) {
                        *reinterpret_cast<float4*>(srow) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        *nq = 0;
                        continue;
                    }
                    const int r = r0 - 1 + rl;
                    const bool own = rl >= 1 && rl <= rows_here;
                    const int blo = own ? (int)kMagicBits : trash_bits;
                    const int bhi = own ? max_bits : trash_bits;
                    const float ncma = cmt[rl * p.units_per_row + uca];
                    const float ncmb = cmt[rl * p.units_per_row + ucb];
                    const float2 d01 = __fadd2_rn(raw_pair(rr[j].x), make_float2(pp[j].x, pp[j].y));
                    const float2 d23 = __fadd2_rn(raw_pair(rr[j].y), make_float2(pp[j].z, pp[j].w));
                    const float2 n01 = make_float2(split > 0 ? ncma : ncmb, split > 1 ? ncma : ncmb);
                    const float2 n23 = make_float2(split > 2 ? ncma : ncmb, split > 3 ? ncma : ncmb);
                    float2 c01 = __fadd2_rn(d01, n01), c23 = __fadd2_rn(d23, n23);
                    if (STACKED) {
                        const float ncr = crt[rl];
                        c01 = __fadd2_rn(__fadd2_rn(c01, make_float2(ncr, ncr)),
                                         make_float2(ncc[0], ncc[1]));
                        c23 = __fadd2_rn(__fadd2_rn(c23, make_float2(ncr, ncr)),
                                         make_float2(ncc[2], ncc[3]));
                    }
                    const float2 e01 = __fmul2_rn(c01, make_float2(gg[j].x, gg[j].y));
                    const float2 e23 = __fmul2_rn(c23, make_float2(gg[j].z, gg[j].w));
                    const float2 iw = make_float2(p.hist_inv_w, p.hist_inv_w);
                    const float2 nl = make_float2(p.hist_neg_lo_s, p.hist_neg_lo_s);
                    const float2 mgc = make_float2(kMagic, kMagic);
                    const float2 u01 = __fadd2_rd(__ffma2_rn(e01, iw, nl), mgc);
                    const float2 u23 = __fadd2_rd(__ffma2_rn(e23, iw, nl), mgc);
                    atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u01.x), blo), bhi) - kMagicBits], 1u);
                    atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u01.y), blo), bhi) - kMagicBits], 1u);
                    atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u23.x), blo), bhi) - kMagicBits], 1u);
                    atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u23.y), blo), bhi) - kMagicBits], 1u);
                    const float e[4] = {e01.x, e01.y, e23.x, e23.y};
                    float sv[4];
                    uint32_t bits = 0;
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        sv[i] = e[i] > p.zero_thr ? e[i] : 0.0f;
                        bits |= (uint32_t)(sv[i] > 0.0f) << i;
                    }
                    *reinterpret_cast<float4*>(srow) = make_float4(sv[0], sv[1], sv[2], sv[3]);
                    *nq = (uint8_t)bits;
                    if (bits) {
                        // signal at row rl, s-tile column x lies in the
                        // windows of own rows rl-2 .. rl+1, columns x-2 ..
                        // x+2: an 8-bit run from column col + 2
                        const uint32_t run = bits | bits << 1 | bits << 2 | bits << 3 | bits << 4;
                        const uint32_t x0 = (uint32_t)col + 2, w = x0 >> 5, sh = x0 & 31;
                        const uint32_t lo = run << sh, hi = sh > 24 ? run >> (32 - sh) : 0u;
                        for (int rr = max(1, rl - 2); rr <= min(rows_here, rl + 1); rr++) {
                            atomicOr(&cbits[rr * WPR + w], lo);
                            if (hi) atomicOr(&cbits[rr * WPR + w + 1], hi);
                        }
                    }
                    if (own && out.corrected) {
                        const uint32_t off = (uint32_t)r * p.cols + (uint32_t)col;
                        float* dst = out.corrected + (size_t)f * p.frame_px + mod_base + off;
                        *reinterpret_cast<float4*>(dst) = make_float4(e[0], e[1], e[2], e[3]);
                    }
                }
            }
        }
        // the next tile's common mode, in flight during the rest of this one
        if (t + gridDim.x < n_tiles && tid < ncmt) cmv = tile_cm(t + gridDim.x, tid);
        __syncthreads();

        // 2. the marked pixels into a list (a warp scan and one shared
        //    atomic per warp reserve each thread's slots; list order is
        //    free), clearing the bitmap for the next tile
        const uint32_t n_words = (uint32_t)rows_here * WPR;
        for (uint32_t base = 0; base < n_words; base += nthr) {
            const uint32_t q = base + tid;
            uint32_t word = 0;
            int rl = 0, x0 = 0;
            if (q < n_words) {
                rl = 1 + (int)(q / WPR);
                x0 = 32 * (int)(q % WPR);
                uint32_t* cw = cbits + rl * WPR + (q % WPR);
                word = *cw;
                *cw = 0;
                // keep s-tile columns 4 .. C + 3 (real columns 0 .. C - 1)
                if (x0 < 4) word &= 0xFFFFFFFFu << (4 - x0);
                const int xe = C + 4 - x0;
                if (xe < 32) word &= xe > 0 ? 0xFFFFFFFFu >> (32 - xe) : 0u;
            }
            const unsigned wm = __activemask();
            const uint32_t cnt = (uint32_t)__popc(word);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(wm, incl, o);
                if (lane >= o) incl += v;
            }
            const int wl = 31 - __clz((int)wm);
            const uint32_t tot = __shfl_sync(wm, incl, wl);
            uint32_t at0 = 0;
            if (lane == wl && tot) at0 = atomicAdd(&s_nc, tot);
            at0 = __shfl_sync(wm, at0, wl);
            uint32_t at = at0 + incl - cnt;
            while (word && at < kMbCap) {
                const int bit = __ffs(word) - 1;
                word &= word - 1;
                list[at++] = ((uint32_t)rl << 16) | (uint32_t)(x0 + bit - 4);
            }
        }
        __syncthreads();

        // 3. the bank at the listed pixels (every own pixel if the list
        //    overflowed): first the valid features of each, then, for the
        //    few with some valid feature (a second list), the sums and the
        //    hit, so that the sums run with every lane on such a pixel
        const uint32_t n_list = s_nc;
        const bool scan = n_list > kMbCap;
        const uint32_t n_work = scan ? (uint32_t)rows_here * (uint32_t)C : n_list;
        // (row, column) of work item j, and its window mask: rows rl-1 ..
        // rl+2, columns c-2 .. c+2 are bits 2 + c % 4 .. 6 + c % 4 of
        // nibbles c / 4 .. c / 4 + 2
        auto item_at = [&](uint32_t j, int& rl, int& c) {
            if (scan) {
                rl = 1 + (int)(j / (uint32_t)C);
                c = (int)(j % (uint32_t)C);
            } else {
                const uint32_t e = list[j];
                rl = (int)(e >> 16);
                c = (int)(e & 0xFFFFu);
            }
        };
        auto window = [&](int rl, int c) -> uint32_t {
            const uint8_t* nw = nib + (rl - 1) * NQ + c / 4;
            const int sh = 2 + (c & 3);
            uint32_t win = 0;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint8_t* g = nw + i * NQ;
                const uint32_t gr = (uint32_t)g[0] | (uint32_t)g[1] << 4 | (uint32_t)g[2] << 8;
                win |= ((gr >> sh) & 0x1Fu) << (5 * i);
            }
            return win;
        };
        if (!scan) {
            for (uint32_t base = 0; base < n_work; base += nthr) {
                const uint32_t j = base + tid;
                uint32_t valid = 0;
                if (j < n_work) {
                    int rl, c;
                    item_at(j, rl, c);
                    const uint32_t win = window(rl, c);
                    if (win) valid = valid_features(sb, stile + (rl - 1) * P + c + 2, win);
                }
                const unsigned wm = __activemask();
                const uint32_t bal = __ballot_sync(wm, valid != 0);
                if (bal) {
                    const int lead = __ffs(bal) - 1;
                    uint32_t at0 = 0;
                    if (lane == lead) at0 = atomicAdd(&s_nv, (uint32_t)__popc(bal));
                    at0 = __shfl_sync(wm, at0, lead);
                    if (valid) vlist[at0 + __popc(bal & ((1u << lane) - 1u))] = j | valid << 24;
                }
            }
            __syncthreads();
            const uint32_t n_valid = s_nv;
            for (uint32_t base = 0; base < n_valid; base += nthr) {
                const uint32_t k = base + tid;
                bool emit = false;
                pd_hit h;
                uint32_t n = 0, pix = 0;
                if (k < n_valid) {
                    const uint32_t e = vlist[k];
                    int rl, c;
                    item_at(e & 0xFFFFFFu, rl, c);
                    float E, dx, dy;
                    uint32_t npix;
                    sum_features(sb, stile + (rl - 1) * P + c + 2, e >> 24, E, dx, dy, npix);
                    if (E != 0.0f)
                        emit = make_hit(p, hhit, E, dx, dy, npix, r0 - 1 + rl, c, frame_base + f,
                                        mod_base, h, n, pix);
                }
                emit_hits(p, out, emit, h, n, pix, lane, __activemask());
            }
        } else {
            for (uint32_t base = 0; base < n_work; base += nthr) {
                const uint32_t j = base + tid;
                bool emit = false;
                pd_hit h;
                uint32_t n = 0, pix = 0;
                if (j < n_work) {
                    int rl, c;
                    item_at(j, rl, c);
                    const uint32_t win = window(rl, c);
                    const float* w = stile + (rl - 1) * P + c + 2;
                    const uint32_t valid = win ? valid_features(sb, w, win) : 0u;
                    if (valid) {
                        float E, dx, dy;
                        uint32_t npix;
                        sum_features(sb, w, valid, E, dx, dy, npix);
                        if (E != 0.0f)
                            emit = make_hit(p, hhit, E, dx, dy, npix, r0 - 1 + rl, c,
                                            frame_base + f, mod_base, h, n, pix);
                    }
                }
                emit_hits(p, out, emit, h, n, pix, lane, __activemask());
            }
        }
        __syncthreads();
        if (prefetcher && t + 2 * step < n_tiles) {
            TileWalk nx = walk;
            nx.next();
            nx.next();
            prefetch_tile_rows(raw, nx, bc.rb, p.rows, p.cols, p.frame_px, 2);
        }
    }
    for (uint32_t b = tid; b < p.hist_bins; b += nthr) {
        if (hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)hpix[b]);
        if (hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)hhit[b]);
    }
}

// Valid features of every window mask of an all-binary bank (no tap is
// read: the tests are mask tests and popcounts).
__global__ void vtab_kernel(const MatchedBank* __restrict__ bank, uint8_t* __restrict__ vtab) {
    const uint32_t win = blockIdx.x * blockDim.x + threadIdx.x;
    if (win >= (1u << 20)) return;
    uint32_t valid = 0;
    for (uint32_t ft = 0; ft < bank->n_features; ft++)
        if ((win & bank->m0[ft]) == 0 && (float)__popc(win & bank->m1[ft]) >= bank->nmin[ft])
            valid |= 1u << ft;
    vtab[win] = (uint8_t)valid;
}

// Nonzero taps of one 4 x 5 filter, row-major, appended to list.
void compile_taps(const float (*flt)[5], MatchedTap* list, uint32_t* n) {
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 5; j++)
            if (flt[i][j] != 0.0f) {
                list[*n].i = (uint8_t)i;
                list[*n].j = (uint8_t)j;
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
    mb.all_binary = 1;
    for (uint32_t f = 0; f < b.n_features; f++)
        if (!mb.f1_unit[f] || !mb.f0_pos[f]) mb.all_binary = 0;
    mb.vtab = nullptr;
    mb.off1[b.n_features] = (uint16_t)n1;
    mb.off0[b.n_features] = (uint16_t)n0;
    mb.offx[b.n_features] = (uint16_t)nx;
    mb.offy[b.n_features] = (uint16_t)ny;
    *out = mb;
    return true;
}

cudaError_t build_vtab(const MatchedBank* bank_dev, uint8_t* vtab) {
    vtab_kernel<<<(1u << 20) / 256, 256>>>(bank_dev, vtab);
    cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : cudaDeviceSynchronize();
}

// Band form of the matched stencil: single gain, raw - pedestal before the
// common mode, four-pixel chunks (as the band stencil's), and bands of at
// least one row within about 100 KB of shared memory.
static bool matched_band_config(const ChainParams& p, BandConfig* out) {
    if (cm_after_gain(p)) return false;
    BandConfig bc = make_band_config(p);
    if (!bc.ok || bc.vec != 4) return false;
    uint32_t rb = std::min<uint32_t>(std::max<uint32_t>(4, 12288 / p.cols), p.rows);
    while (rb > 1 && band_smem(p, rb, bc.pitch) > 100 * 1024) rb--;
    if (band_smem(p, rb, bc.pitch) > 100 * 1024) return false;
    bc.rb = rb;
    bc.n_bands = (p.rows + rb - 1) / rb;
    *out = bc;
    return true;
}

static int g_attr_dev_mband = -1;

cudaError_t launch_matched(const ChainParams& p, const MatchedBank* bank_dev,
                           const uint16_t* raw, uint32_t n_frames, uint32_t frame_base,
                           const CallOut& out, cudaStream_t stream, const MultiGain* mg) {
    BandConfig bc;
    if (!mg && matched_band_config(p, &bc)) {
        const unsigned long long n_tiles =
            (unsigned long long)n_frames * p.n_modules * bc.n_bands;
        if (n_tiles == 0) return cudaSuccess;
        int dev = 0;
        cudaGetDevice(&dev);
        if (g_attr_dev_mband != dev) {
            for (auto k : {matched_band_kernel<false>, matched_band_kernel<true>}) {
                cudaError_t e = cudaFuncSetAttribute(
                    k, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
                if (e != cudaSuccess) return e;
            }
            g_attr_dev_mband = dev;
        }
        const size_t smem = band_smem(p, bc.rb, bc.pitch);
        const size_t per_cta = smem + sizeof(MatchedBank) + 1024;
        int per_sm = (int)((228 * 1024) / per_cta);
        per_sm = std::max(1, std::min(per_sm, 2));
        unsigned long long grid = (unsigned long long)device_sm_count() * per_sm;
        if (grid > n_tiles) grid = n_tiles;
        const unsigned threads = bc.tx * bc.ty;
        if (cm_kind(p) == PD_CM_MEAN_STACKED)
            matched_band_kernel<true><<<(unsigned)grid, threads, smem, stream>>>(
                p, bank_dev, raw, frame_base, out, bc, n_tiles);
        else
            matched_band_kernel<false><<<(unsigned)grid, threads, smem, stream>>>(
                p, bank_dev, raw, frame_base, out, bc, n_tiles);
        return cudaGetLastError();
    }
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
