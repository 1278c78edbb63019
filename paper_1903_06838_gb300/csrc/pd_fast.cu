// pd_fast.cu — throughput kernels of the chain.
//
//   cm_big_kernel      common mode of one large unit (a bank of thousands of
//                      pixels) per CTA (paper section "Common Mode", Fig. c;
//                      the estimator is the lower median over d < cut).
//                      Pass A histograms d into 4096 bins of 1/8 ADU whose
//                      window [cut - 512, cut) ends exactly at the cut, keeping
//                      every pixel's 16-bit bin code in shared memory.  The
//                      bin holding rank floor((n-1)/2) is found by a scan;
//                      pass B gathers that bin's pixels (recomputing their d
//                      from L2-resident raw and pedestal) and an exact radix
//                      select over them gives the median.  When the median
//                      falls in the window's open-ended bottom bin, or the
//                      bin holds more candidates than the buffer, the CTA
//                      selects over the whole unit instead (same result).
//   stencil_band_kernel  dark, common mode, gain (Fig. b), zeroing, 3x3 local
//                      maximum, charge sum, count (Fig. e), centroid (Fig. f),
//                      hits and summaries for a band of full-width rows of a
//                      module.  Each thread owns one 4-pixel column chunk for
//                      all rows of the band, so its unit/column bookkeeping is
//                      computed once.  The zeroed signal of the band and its
//                      two halo rows is staged in shared memory; seed
//                      candidates are compacted into a list before the 3x3
//                      work.
//
// Bin codes use the floor-by-magic-number identity: for |t| < 2^22,
// fadd_rd(t, 1.5*2^23) has bit pattern 0x4B400000 + floor(t), and a fused
// multiply-add rounded down computes floor(8*(d - lo)) exactly when 8*lo is an
// integer (8*d is exact).  All arithmetic on values that reach an output is
// round-to-nearest in the chain's order (compiled with --fmad=false).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_cm_generic.cuh"
#include "pd_dev.cuh"
#include "pd_fast.cuh"

// rows of loads a thread keeps in flight (common mode, band stencil)
#ifndef PD_CM_UNROLL
#define PD_CM_UNROLL 8
#endif
#ifndef PD_BAND_UNROLL
#define PD_BAND_UNROLL 2
#endif


namespace pd {

namespace {

// ---------------------------------------------------------------------------
// Common mode of large units.
struct CmBigShared {
    uint32_t gsum[kCmBins / 32];
    uint32_t swarp[32];
    uint32_t s_bin, s_rank, s_n, s_cand, s_prefix, s_rrank;
};

// Common mode of unit `item` (= frame * units_per_frame + unit) into
// cm_out[item]; cm_smem: cm_big_smem_bytes(p) of dynamic shared memory.
// MG: auto-ranging words; a word with a bit of stage_mask set is not in
// stage 0 and stays out of the set (a stage-0 word is its own ADC value).
template <int VEC, bool MG = false>
__device__ void cm_big_unit(const ChainParams& p, const uint16_t* __restrict__ raw,
                            float* __restrict__ cm_out, const CmBigConfig& cfg, uint32_t item,
                            uint32_t* cm_smem, CmBigShared& sh, uint32_t stage_mask = 0) {
    uint32_t* hist = cm_smem;                            // kCmBins + spare + pad
    float* cand = reinterpret_cast<float*>(hist + kCmBins + 4);  // kCandCap
    uint32_t* codes = reinterpret_cast<uint32_t*>(cand + kCandCap);  // VEC=2: pairs
    uint32_t* gsum = sh.gsum;
    uint32_t &s_bin = sh.s_bin, &s_rank = sh.s_rank, &s_n = sh.s_n, &s_cand = sh.s_cand;
    uint32_t &s_prefix = sh.s_prefix, &s_rrank = sh.s_rrank;

    const uint32_t f = item / p.units_per_frame;
    const uint32_t u = item % p.units_per_frame;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
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
    const float* npm = p.nped + mod_base;
    const uint32_t TX = cfg.tx, TY = cfg.ty;
    const uint32_t tx = tid % TX, ty = tid / TX;
    const bool active = ty < TY;

    // VEC == 2: all raw pairs of the unit are copied into the code buffer
    // at once (one request per pair, none held in registers), before the
    // histogram is zeroed so the copies' latency overlaps it; each pair is
    // replaced in place by its two bin codes in pass A
    if (VEC == 2 && active) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(fr + (r0 + ty) * p.cols + c0) + tx;
        const uint32_t sstride = TY * p.cols / 2;
        uint32_t* dst = codes + ty * TX + tx;
        for (uint32_t r = ty; r < p.unit_rows; r += TY) {
            cp_async4(dst, src);
            src += sstride;
            dst += TY * TX;
        }
    }
    for (uint32_t i = tid; i < kCmBins / 4; i += nthr)
        reinterpret_cast<uint4*>(hist)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        s_cand = 0;
        hist[kCmBins] = 0;
    }
    __syncthreads();

    // pass A: histogram of bin codes, codes kept for pass B.  Loads of U
    // rows are issued before any of them is used, to keep several memory
    // requests of every thread in flight.  Every pixel does one atomic: a
    // pixel with d >= cut adds to the spare bin kCmBins, which is never read.
    if (active) {
        if (VEC == 2) {
            cp_async_wait_all();  // each thread reads back only its own copies
            constexpr int U = PD_CM_UNROLL;
            const float2* prow = reinterpret_cast<const float2*>(npm + (r0 + ty) * p.cols + c0) + tx;
            const uint32_t stride = TY * p.cols / 2;  // pairs between a thread's rows
            uint32_t* cptr = codes + ty * TX + tx;
            const uint32_t cstride = TY * TX;
            const float2 eight = make_float2(8.0f, 8.0f);
            const float2 mw = make_float2(cfg.magic_w, cfg.magic_w);
            uint32_t r = ty;
            for (; r + (U - 1) * TY < p.unit_rows; r += U * TY) {
                float2 pp[U];
#pragma unroll
                for (int j = 0; j < U; j++) pp[j] = prow[j * stride];
#pragma unroll
                for (int j = 0; j < U; j++) {
                    const uint32_t x = cptr[j * cstride];
                    const float2 d = __fadd2_rn(raw_pair(x), pp[j]);
                    const float2 u = __ffma2_rd(d, eight, mw);
                    int b0 = min(max(__float_as_int(u.x), (int)kMagicBits),
                                 (int)(kMagicBits + kCmBins));
                    int b1 = min(max(__float_as_int(u.y), (int)kMagicBits),
                                 (int)(kMagicBits + kCmBins));
                    if (MG) {
                        if (x & stage_mask) b0 = (int)(kMagicBits + kCmBins);
                        if ((x >> 16) & stage_mask) b1 = (int)(kMagicBits + kCmBins);
                    }
                    atomicAdd(&hist[(uint32_t)b0 - kMagicBits], 1u);
                    atomicAdd(&hist[(uint32_t)b1 - kMagicBits], 1u);
                    cptr[j * cstride] = __byte_perm((uint32_t)b0, (uint32_t)b1, 0x5410u);
                }
                prow += U * stride;
                cptr += U * cstride;
            }
            for (; r < p.unit_rows; r += TY) {
                const uint32_t x = *cptr;
                const float2 d = __fadd2_rn(raw_pair(x), *prow);
                const float2 u = __ffma2_rd(d, eight, mw);
                int b0 = min(max(__float_as_int(u.x), (int)kMagicBits),
                             (int)(kMagicBits + kCmBins));
                int b1 = min(max(__float_as_int(u.y), (int)kMagicBits),
                             (int)(kMagicBits + kCmBins));
                if (MG) {
                    if (x & stage_mask) b0 = (int)(kMagicBits + kCmBins);
                    if ((x >> 16) & stage_mask) b1 = (int)(kMagicBits + kCmBins);
                }
                atomicAdd(&hist[(uint32_t)b0 - kMagicBits], 1u);
                atomicAdd(&hist[(uint32_t)b1 - kMagicBits], 1u);
                *cptr = __byte_perm((uint32_t)b0, (uint32_t)b1, 0x5410u);
                prow += stride;
                cptr += cstride;
            }
        } else {
            uint32_t off = (r0 + ty) * p.cols + c0 + tx;
            for (uint32_t r = ty; r < p.unit_rows; r += TY, off += TY * p.cols) {
                const uint32_t w = fr[off];
                const float d = __fadd_rn(__uint2float_rn(w), npm[off]);
                uint32_t k = cm_code(d, cfg.magic_w);
                k = min(k, kCmBins);
                if (MG && (w & stage_mask)) k = kCmBins;
                atomicAdd(&hist[k], 1u);
                reinterpret_cast<uint16_t*>(codes)[r * TX + tx] = (uint16_t)k;
            }
        }
    }
    __syncthreads();

    // locate rank floor((n-1)/2) of the values below the cut
    const uint32_t min_count = p.cm_min_count;
    find_rank<kCmBins>(
        hist,
        [min_count](uint32_t total) {
            return (total > 0 && total >= min_count) ? (total - 1) / 2 : total;
        },
        gsum, &s_n, &s_bin, &s_rank);
    const uint32_t n = s_n;
    if (n == 0 || n < min_count) {
        if (tid == 0) cm_out[item] = 0.0f;
        return;
    }
    const uint32_t bin = s_bin, brank = s_rank;

    // the key of pixel i of the unit (kSent when d >= cut)
    auto unit_key = [&](uint32_t i) -> uint32_t {
        const uint32_t off = (r0 + i / p.unit_cols) * p.cols + c0 + i % p.unit_cols;
        const uint32_t w = fr[off];
        if (MG && (w & stage_mask)) return kSent;
        const float d = __fadd_rn(__uint2float_rn(w), npm[off]);
        return d < p.cm_cut ? order_key(d) : kSent;
    };

    if (bin != 0) {
        // pass B: positions of the winning bin's pixels (shared memory only),
        // then one parallel fetch of their raw value and pedestal.  The codes
        // are a row-major array of one 16-bit code per pixel of the unit (in
        // both layouts), read eight at a time; a halfword h of y = word ^
        // (bin, bin) is zero iff bit 15 of ((h & 0x7FFF) + 0x7FFF) | h is
        // clear.  About one pixel in a hundred matches: each takes a slot
        // with a shared atomic (list order is free; s_cand counts every
        // match, so an overflow is seen).
        uint32_t* cidx = reinterpret_cast<uint32_t*>(cand);
        const uint32_t both = bin | (bin << 16);
        auto take = [&](uint32_t y, uint32_t px0) {
            uint32_t z = ~((((y & 0x7FFF7FFFu) + 0x7FFF7FFFu) | y)) & 0x80008000u;
            while (z) {
                const uint32_t at = atomicAdd(&s_cand, 1u);
                if (at < kCandCap) cidx[at] = px0 + ((z & 0x8000u) ? 0u : 1u);
                z &= z - 1;
            }
        };
        const uint32_t n8 = p.unit_px / 8;
        const uint4* c8 = reinterpret_cast<const uint4*>(codes);
        for (uint32_t q = tid; q < n8; q += nthr) {
            const uint4 v = c8[q];
            const uint32_t y0 = v.x ^ both, y1 = v.y ^ both, y2 = v.z ^ both, y3 = v.w ^ both;
            const uint32_t t0 = ((y0 & 0x7FFF7FFFu) + 0x7FFF7FFFu) | y0;
            const uint32_t t1 = ((y1 & 0x7FFF7FFFu) + 0x7FFF7FFFu) | y1;
            const uint32_t t2 = ((y2 & 0x7FFF7FFFu) + 0x7FFF7FFFu) | y2;
            const uint32_t t3 = ((y3 & 0x7FFF7FFFu) + 0x7FFF7FFFu) | y3;
            if ((t0 & t1 & t2 & t3 & 0x80008000u) != 0x80008000u) {
                take(y0, 8 * q);
                take(y1, 8 * q + 2);
                take(y2, 8 * q + 4);
                take(y3, 8 * q + 6);
            }
        }
        const uint16_t* c16 = reinterpret_cast<const uint16_t*>(codes);
        for (uint32_t i = 8 * n8 + tid; i < p.unit_px; i += nthr)
            if (c16[i] == bin) {
                const uint32_t at = atomicAdd(&s_cand, 1u);
                if (at < kCandCap) cidx[at] = i;
            }
        __syncthreads();
        const uint32_t mc = s_cand;
        if (mc <= kCandCap) {
            // position i (row-major in the unit) -> d, in place
            for (uint32_t t = tid; t < mc; t += nthr) {
                const uint32_t i = cidx[t];
                const uint32_t off = (r0 + i / p.unit_cols) * p.cols + c0 + i % p.unit_cols;
                cand[t] = __fadd_rn(__uint2float_rn(fr[off]), npm[off]);
            }
            __syncthreads();
            // exact select inside the bin: 1024 sub-bins of 1/8192 ADU (d - lo
            // rounded to nearest is monotone in d, so sub-bins stay ordered),
            // then the few values of the target sub-bin are ranked by counting
            const float lo_b = __fadd_rn(cfg.w_lo, __fmul_rn((float)bin, 0.125f));
            uint32_t* sub = hist;  // reuse: 1024 sub-bins
            for (uint32_t i = tid; i < 1024 / 4; i += nthr)
                reinterpret_cast<uint4*>(sub)[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
            for (uint32_t t = tid; t < mc; t += nthr) {
                const float x = __fmul_rn(__fsub_rn(cand[t], lo_b), 8192.0f);
                const uint32_t sb = min((uint32_t)max(__float2int_rd(x), 0), 1023u);
                codes[t] = sb;  // codes are no longer needed: keep each sub-bin
                atomicAdd(&sub[sb], 1u);
            }
            __syncthreads();
            find_rank<1024>(
                sub, [brank](uint32_t) { return brank; }, gsum, &s_prefix, &s_bin, &s_rank);
            const uint32_t sbin = s_bin, srank = s_rank;
            // values of the target sub-bin, then rank by counting among them
            float* few = reinterpret_cast<float*>(sub + 1024);
            if (tid == 0) s_rrank = 0;
            __syncthreads();
            for (uint32_t t = tid; t < mc; t += nthr)
                if (codes[t] == sbin) few[atomicAdd(&s_rrank, 1u)] = cand[t];
            __syncthreads();
            const uint32_t nf = s_rrank;
            for (uint32_t t = tid; t < nf; t += nthr) {
                const uint32_t kt = order_key(few[t]);
                uint32_t less = 0, leq = 0;
                for (uint32_t j = 0; j < nf; j++) {
                    const uint32_t kj = order_key(few[j]);
                    less += kj < kt;
                    leq += kj <= kt;
                }
                if (less <= srank && srank < leq) cm_out[item] = few[t];
            }
            return;
        }
    }
    // whole-unit exact selection (bottom bin or candidate overflow)
    const uint32_t key = block_radix_select(unit_key, p.unit_px, (n - 1) / 2, hist,
                                            &s_prefix, &s_rrank);
    if (tid == 0) cm_out[item] = key_value(key);
}

template <int VEC, bool MG>
__global__ void __launch_bounds__(512, 2)
    cm_big_kernel(ChainParams p, const uint16_t* __restrict__ raw,
                  float* __restrict__ cm_out, CmBigConfig cfg, uint32_t stage_mask) {
    extern __shared__ __align__(16) uint32_t cm_smem[];
    __shared__ CmBigShared sh;
    cm_big_unit<VEC, MG>(p, raw, cm_out, cfg, blockIdx.x, cm_smem, sh, stage_mask);
}

// ---------------------------------------------------------------------------
// Common mode of small units (at most kRowMaxPx pixels, e.g. 384-pixel ASIC
// rows): one warp per unit, every pixel of the unit in the lanes' registers.
// Level 1: 256 bins of 1 ADU from w0 = min(cut - 256, -128) in warp-private
// shared memory (d < w0 in bin 0, d in [w0 + 255, cut) in bin 255, d >= cut
// in the spare bin 256), a warp scan finds the bin of rank floor((n-1)/2).
// The window stays around zero, where dark-subtracted values and their
// median lie, also when the cut is far above 128 ADU.  Level 2: the bin's
// values into 64 sub-bins of 1/64 ADU (RN(d - lo) is monotone in d), scan
// again.  Level 3: the few values of that sub-bin, ranked by counting.  A
// median in bin 0 (open below) or in an open bin 255 goes to a warp-level
// 4-pass radix select over the unit.
constexpr int kRowMaxPx = 512;      // pixels per unit handled by one warp
constexpr int kRowPerLane = kRowMaxPx / 32;
constexpr int kRowWarps = 8;        // units per CTA
struct __align__(16) RowWarpShared {
    uint32_t hist[256 + 4];  // then sub: both zeroed as one run of 16-byte words
    uint32_t sub[64];
    float few[64];
    uint32_t n_few;
};
static_assert(sizeof(uint32_t) * (256 + 4) % 16 == 0, "sub follows hist on a 16-byte boundary");

// warp inclusive scan of one value per lane
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += x;
    }
    return v;
}

// Locate rank k among the bins of a warp, lane l holding bins l * PER ..
// l * PER + PER - 1 in loc with the exclusive and inclusive warp prefix of
// their counts: *bin and the rank within it; false when k >= total.
template <int PER>
__device__ __forceinline__ bool warp_locate(const uint32_t (&loc)[PER], uint32_t excl,
                                            uint32_t incl, uint32_t k, int lane, uint32_t* bin,
                                            uint32_t* krem) {
    const bool mine = excl <= k && k < incl;
    uint32_t b = 0, r = 0;
    if (mine) {
        uint32_t below = excl;
#pragma unroll
        for (int j = 0; j < PER; j++) {
            if (below + loc[j] > k) {
                b = lane * PER + j;
                r = k - below;
                break;
            }
            below += loc[j];
        }
    }
    const uint32_t who = __ballot_sync(0xffffffffu, mine);
    if (!who) return false;
    const int src = __ffs(who) - 1;
    *bin = __shfl_sync(0xffffffffu, b, src);
    *krem = __shfl_sync(0xffffffffu, r, src);
    return true;
}

// Locate rank k among bins hist[0..nb) (nb = 32 * per): *bin and the rank
// within it; returns false when k >= total.
template <int PER>
__device__ __forceinline__ bool warp_find_rank(const uint32_t* hist, uint32_t k, int lane,
                                               uint32_t* bin, uint32_t* krem) {
    uint32_t loc[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; j++) {
        loc[j] = hist[lane * PER + j];
        sum += loc[j];
    }
    const uint32_t incl = warp_incl_scan(sum, lane);
    return warp_locate<PER>(loc, incl - sum, incl, k, lane, bin, krem);
}

// Common mode of unit `item` by one whole warp (lane = lane index).
// PER: pixels per lane the unit can hold (PER * 32 >= unit_px; a multiple of 4).
template <int PER = kRowPerLane>
__device__ void cm_rows_unit(const ChainParams& p, const uint16_t* __restrict__ raw,
                             float* __restrict__ cm_out, unsigned long long item,
                             float magic_1, RowWarpShared& S) {
    const int lane = threadIdx.x & 31;
    // (32-bit division where the item index allows it: the 64-bit one is a
    // long instruction sequence, paid once per 384-pixel unit)
    uint32_t f, u;
    if (item < (1ull << 32)) {
        f = (uint32_t)item / p.units_per_frame;
        u = (uint32_t)item - f * p.units_per_frame;
    } else {
        f = (uint32_t)(item / p.units_per_frame);
        u = (uint32_t)(item - (unsigned long long)f * p.units_per_frame);
    }
    if (cm_kind(p) == PD_CM_NONE) {
        if (lane == 0) cm_out[item] = 0.0f;
        return;
    }
    const uint32_t m = u / p.units_per_module;
    const uint32_t um = u - m * p.units_per_module;
    const uint32_t ur = p.units_per_row == 1 ? um : um / p.units_per_row;
    const uint32_t r0 = ur * p.unit_rows;
    const uint32_t c0 = (um - ur * p.units_per_row) * p.unit_cols;
    const size_t mod_base = (size_t)m * p.module_px;
    const uint16_t* fr = raw + (size_t)f * p.frame_px + mod_base;
    const float* npm = p.nped + mod_base;
    const uint32_t npx = p.unit_px;

    for (int i = lane; i < (256 + 4 + 64) / 4; i += 32)
        reinterpret_cast<uint4*>(S.hist)[i] = make_uint4(0, 0, 0, 0);
    if (lane == 0) S.n_few = 0;
    __syncwarp();

    // d of this lane's pixels: pixel i of the unit = lane + 32 * j, or for
    // aligned single-row units 4 consecutive pixels per load (chunk
    // lane + 32 * (j / 4), pixel 4 * chunk + j % 4)
    float d[PER];
    uint32_t code[PER];
    const bool vec4 = p.unit_rows == 1 && npx % 4 == 0 && c0 % 4 == 0 && p.cols % 4 == 0;
    if (vec4) {
        const uint16_t* rrow = fr + r0 * p.cols + c0;
        const float* prow = npm + r0 * p.cols + c0;
#pragma unroll
        for (int jc = 0; jc < PER / 4; jc++) {
            const uint32_t ch = lane + 32 * jc;
            uint2 rw = make_uint2(0, 0);
            float4 pp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (4 * ch < npx) {
                rw = *reinterpret_cast<const uint2*>(rrow + 4 * ch);
                pp = *reinterpret_cast<const float4*>(prow + 4 * ch);
            }
            const float2 d01 = __fadd2_rn(raw_pair(rw.x), make_float2(pp.x, pp.y));
            const float2 d23 = __fadd2_rn(raw_pair(rw.y), make_float2(pp.z, pp.w));
            const float dv[4] = {d01.x, d01.y, d23.x, d23.y};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int j = 4 * jc + q;
                d[j] = 0.0f;
                code[j] = 256;
                if (4 * ch < npx) {
                    d[j] = dv[q];
                    int b = __float_as_int(__fmaf_rd(d[j], 1.0f, magic_1));
                    b = min(max(b, (int)kMagicBits), (int)(kMagicBits + 255));
                    code[j] = d[j] < p.cm_cut ? (uint32_t)b - kMagicBits : 256u;
                    atomicAdd(&S.hist[code[j]], 1u);
                }
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < PER; j++) {
            const uint32_t i = lane + 32 * j;
            d[j] = 0.0f;
            code[j] = 256;
            if (i < npx) {
                const uint32_t off = p.unit_rows == 1
                                         ? r0 * p.cols + c0 + i
                                         : (r0 + i / p.unit_cols) * p.cols + c0 + i % p.unit_cols;
                d[j] = __fadd_rn(__uint2float_rn(fr[off]), npm[off]);
                int b = __float_as_int(__fmaf_rd(d[j], 1.0f, magic_1));
                b = min(max(b, (int)kMagicBits), (int)(kMagicBits + 255));
                code[j] = d[j] < p.cm_cut ? (uint32_t)b - kMagicBits : 256u;
                atomicAdd(&S.hist[code[j]], 1u);
            }
        }
    }
    __syncwarp();
    // the lane's eight bins (two 16-byte reads) and their warp scan: n =
    // values below the cut (every bin but the spare one), then the bin of
    // rank floor((n-1)/2)
    uint32_t loc[8];
    {
        const uint4 lo4 = reinterpret_cast<const uint4*>(S.hist)[2 * lane];
        const uint4 hi4 = reinterpret_cast<const uint4*>(S.hist)[2 * lane + 1];
        loc[0] = lo4.x; loc[1] = lo4.y; loc[2] = lo4.z; loc[3] = lo4.w;
        loc[4] = hi4.x; loc[5] = hi4.y; loc[6] = hi4.z; loc[7] = hi4.w;
    }
    uint32_t lsum = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) lsum += loc[j];
    const uint32_t incl = warp_incl_scan(lsum, lane);
    const uint32_t n = __shfl_sync(0xffffffffu, incl, 31);
    if (n == 0 || n < p.cm_min_count) {
        if (lane == 0) cm_out[item] = 0.0f;
        return;
    }
    const uint32_t k = (n - 1) / 2;
    uint32_t bin = 0, kb = 0;
    warp_locate<8>(loc, incl - lsum, incl, k, lane, &bin, &kb);
    // the window's base (magic_1 = 1.5 * 2^23 - w0, both exact) and whether
    // bin 255 is a whole 1-ADU bin (the window ends at the cut)
    const float w0 = __fsub_rn(kMagic, magic_1);
    const bool top_closed = __fadd_rn(w0, 256.0f) == p.cm_cut;
    if (bin != 0 && (bin != 255 || top_closed)) {
        // level 2: sub-bins of the winning 1-ADU bin [lo, lo + 1)
        const float lo = __fadd_rn(w0, (float)bin);
        uint32_t sb[PER];
#pragma unroll
        for (int j = 0; j < PER; j++) {
            sb[j] = 64;
            if (code[j] == bin) {
                const float x = __fmul_rn(__fsub_rn(d[j], lo), 64.0f);
                sb[j] = min((uint32_t)max(__float2int_rd(x), 0), 63u);
                atomicAdd(&S.sub[sb[j]], 1u);
            }
        }
        __syncwarp();
        uint32_t sbin = 0, ks = 0;
        warp_find_rank<2>(S.sub, kb, lane, &sbin, &ks);
        // level 3: values of the winning sub-bin, ranked by counting
#pragma unroll
        for (int j = 0; j < PER; j++)
            if (sb[j] == sbin) {
                const uint32_t slot = atomicAdd(&S.n_few, 1u);
                if (slot < 64) S.few[slot] = d[j];
            }
        __syncwarp();
        const uint32_t nf = S.n_few;
        if (nf <= 64) {
            for (uint32_t t = lane; t < nf; t += 32) {
                const uint32_t kt = order_key(S.few[t]);
                uint32_t less = 0, leq = 0;
                for (uint32_t q = 0; q < nf; q++) {
                    const uint32_t kq = order_key(S.few[q]);
                    less += kq < kt;
                    leq += kq <= kt;
                }
                if (less <= ks && ks < leq) cm_out[item] = S.few[t];
            }
            return;
        }
    }
    // warp radix select over the whole unit (median below the window, or more
    // than 64 values in one sub-bin): 4 passes of 8 bits on IEEE-order keys
    uint32_t prefix = 0, krank = k;
    for (int pass = 0; pass < 4; pass++) {
        const int shift = 24 - 8 * pass;
        for (int i = lane; i < 256; i += 32) S.hist[i] = 0;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < PER; j++) {
            if (code[j] >= 256) continue;  // outside the unit or d >= cut
            const uint32_t key = order_key(d[j]);
            if (pass > 0 && (key >> (shift + 8)) != prefix) continue;
            atomicAdd(&S.hist[(key >> shift) & 255u], 1u);
        }
        __syncwarp();
        uint32_t digit = 0, rem = 0;
        warp_find_rank<8>(S.hist, krank, lane, &digit, &rem);
        prefix = (prefix << 8) | digit;
        krank = rem;
        __syncwarp();
    }
    if (lane == 0) cm_out[item] = key_value(prefix);
}

template <int PER>
__global__ void __launch_bounds__(32 * kRowWarps)
    cm_rows_kernel(ChainParams p, const uint16_t* __restrict__ raw, float* __restrict__ cm_out,
                   unsigned long long n_items, float magic_1) {
    __shared__ RowWarpShared ws[kRowWarps];
    const int w = threadIdx.x >> 5;
    const unsigned long long item = (unsigned long long)blockIdx.x * kRowWarps + w;
    if (item >= n_items) return;  // whole warps only; no block-level barrier follows
    cm_rows_unit<PER>(p, raw, cm_out, item, magic_1, ws[w]);
}

// ---------------------------------------------------------------------------
// Stencil over bands of full-width rows.
struct BandShared {
    uint32_t s_list_n;
    uint32_t swarp[32];
};

// Tiles first, first + step, ... < n_tiles of one call: tile t is band
// t % n_bands of module (t / n_bands) % n_modules of frame t / (n_bands *
// n_modules).  Zeroes this CTA's shared tile and histograms first and adds
// the histograms to the context's at the end.  STACKED: the stacked mean
// common mode, whose module-row and module-column terms follow the units'
// values of each frame and are subtracted after the unit's.  PREFETCH: the
// raw rows of later tiles are asked of L2 ahead of their loads (the
// single-context kernel; the batched one keeps its registers for the items'
// parameters).
template <int VEC, bool STACKED = false, bool MG = false, bool PREFETCH = false>
__device__ void stencil_band_run(const ChainParams& p, const uint16_t* __restrict__ raw,
                                 uint32_t frame_base, const CallOut& out, const BandConfig& bc,
                                 unsigned long long first, unsigned long long n_tiles,
                                 unsigned long long step, uint32_t* band_smem, BandShared& bsh,
                                 const MultiGain& mg = MultiGain{}) {
    const uint32_t P = bc.pitch;                 // floats per s-tile row
    float* stile = reinterpret_cast<float*>(band_smem);          // (rb+2) * P
    uint32_t* hpix = band_smem + (bc.rb + 2) * P;               // hist_bins + spare
    uint32_t* hhit = hpix + p.hist_bins + 4;                     // hist_bins
    uint32_t* list = hhit + p.hist_bins;                         // kSeedCap
    float* cmt = reinterpret_cast<float*>(list + kSeedCap);      // (rb+2) * upr
    float* crt = cmt + (bc.rb + 2) * p.units_per_row;            // (rb+2) row terms
    // seed bitmap: bit c of word row rl marks own pixel (rl, c) above the
    // seed threshold; rows 1 .. rows_here used, zero between tiles
    const uint32_t WPR = (uint32_t)(p.cols + 31) / 32;
    uint32_t* sbits = reinterpret_cast<uint32_t*>(crt + bc.rb + 2);  // (rb+1) x WPR
    uint32_t& s_list_n = bsh.s_list_n;

    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31;
    const int R = (int)p.rows, C = (int)p.cols;
    const uint32_t TX = bc.tx, TY = bc.ty;
    const uint32_t tx = tid % TX, ty = tid / TX;
    const bool active = ty < TY;
    const int col = (int)(tx * VEC);  // first column of this thread's chunk
    // unit columns of the chunk's first and last pixel, and where it splits
    const uint32_t uca = (uint32_t)col / p.unit_cols;
    const uint32_t ucb = (uint32_t)(col + VEC - 1) / p.unit_cols;
    const int split = (int)(ucb * p.unit_cols) - col;  // pixels i >= split use ucb
    const int max_bits = (int)(kMagicBits + p.hist_bins - 1);
    const int trash_bits = (int)(kMagicBits + p.hist_bins);  // spare bin of hpix

    // zero the whole s-tile once (pad columns stay zero), and the histograms
    for (uint32_t i = tid; i < (bc.rb + 2) * P; i += nthr) stile[i] = 0.0f;
    for (uint32_t i = tid; i < 2 * p.hist_bins + 4; i += nthr) hpix[i] = 0;
    for (uint32_t i = tid; i < (bc.rb + 1) * WPR; i += nthr) sbits[i] = 0;
    __syncthreads();

    // negated common mode of (tile row, unit column) entry i of tile tt;
    // each thread holds its entries of the next tile in registers, loaded
    // while the current tile's seeds are tested
    // (tile indices of one call stay below 2^32)
    const uint32_t ncmt = (bc.rb + 2) * p.units_per_row;
    auto tile_cm = [&](uint32_t tt, uint32_t i) -> float {
        const uint32_t fm = tt / bc.n_bands;
        const int r = (int)(tt - fm * bc.n_bands) * (int)bc.rb - 1 + (int)(i / p.units_per_row);
        if (r < 0 || r >= R) return 0.0f;
        // (stacked: each frame's values also hold the row and column terms)
        const size_t fbase = (size_t)fm * p.units_per_module +
                             (STACKED ? (size_t)(fm / p.n_modules) *
                                            (cm_per_frame(p) - p.units_per_frame)
                                      : 0);
        return -out.cm[fbase + ((uint32_t)r / p.unit_rows) * p.units_per_row +
                       i % p.units_per_row];
    };
    float cmv = 0.0f;
    if (first < n_tiles && tid < ncmt) cmv = tile_cm((uint32_t)first, tid);

    TileWalk walk(first, step, bc.n_bands, p.n_modules);
    // the last thread asks L2 for the raw rows (halo rows included) of the
    // next tile now and of the tile after next once a tile is done, so that
    // their loads find them there
    const bool prefetcher = PREFETCH && tid == nthr - 1;
    if (prefetcher && first + step < n_tiles) {
        TileWalk nx = walk;
        nx.next();
        prefetch_tile_rows(raw, nx, bc.rb, p.rows, p.cols, p.frame_px);
    }
    for (unsigned long long t = first; t < n_tiles; t += step, walk.next()) {
        const int band = (int)walk.band;
        const uint32_t m = walk.m, f = walk.f;
        const int r0 = band * (int)bc.rb;
        const int rows_here = min((int)bc.rb, R - r0);
        const size_t mod_base = (size_t)m * p.module_px;
        const uint16_t* fr = raw + (size_t)f * p.frame_px + mod_base;
        const float* npm = p.nped + mod_base;
        const float* gm = p.inv_gain + mod_base;

        // negated common mode of every (tile row, unit column)
        if (tid < ncmt) cmt[tid] = cmv;
        for (uint32_t i = tid + nthr; i < ncmt; i += nthr) cmt[i] = tile_cm((uint32_t)t, i);
        // stacked: negated module-row terms of the tile's rows, and this
        // thread's negated module-column terms
        float ncc[VEC];
        if (STACKED) {
            const float* cmf = out.cm + (size_t)f * cm_per_frame(p) + p.units_per_frame;
            for (uint32_t i = tid; i < bc.rb + 2; i += nthr) {
                const int r = r0 - 1 + (int)i;
                crt[i] = r >= 0 && r < R ? -cmf[(size_t)m * p.rows + r] : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < VEC; i++)
                ncc[i] = active && col + i < C
                             ? -cmf[(size_t)p.n_modules * p.rows + (size_t)m * p.cols + col + i]
                             : 0.0f;
        }
        if (tid == 0) s_list_n = 0;
        __syncthreads();

        // 1. zeroed signal of rows r0-1 .. r0+rows_here (halo rows included);
        //    loads of U rows are issued before any is used.  Halo rows
        //    are not histogrammed: their bins are clamped to the spare bin.
        if (active) {
            const int nrows = rows_here + 2;
            constexpr int U = PD_BAND_UNROLL;
            for (int rl0 = (int)ty; rl0 < nrows; rl0 += U * (int)TY) {
                uint2 rr[U];
                float4 pp[U], gg[U];
                uint16_t r1[U];
                float p1[U], g1[U];
                bool in[U];
#pragma unroll
                for (int j = 0; j < U; j++) {
                    const int rl = rl0 + j * (int)TY;
                    const int r = r0 - 1 + rl;
                    in[j] = rl < nrows && r >= 0 && r < R;
                    const uint32_t off = in[j] ? (uint32_t)r * p.cols + (uint32_t)col : 0u;
                    if (VEC == 4) {
                        if (in[j]) {
                            rr[j] = *reinterpret_cast<const uint2*>(fr + off);
                            pp[j] = *reinterpret_cast<const float4*>(npm + off);
                            gg[j] = *reinterpret_cast<const float4*>(gm + off);
                        }
                    } else {
                        if (in[j]) {
                            r1[j] = fr[off];
                            p1[j] = npm[off];
                            g1[j] = gm[off];
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < U; j++) {
                    const int rl = rl0 + j * (int)TY;
                    if (rl >= nrows) continue;
                    float* srow = stile + rl * P + 4 + col;
                    if (!in[j]) {
#pragma unroll
                        for (int i = 0; i < VEC; i++) srow[i] = 0.0f;
                        continue;
                    }
                    const int r = r0 - 1 + rl;
                    const bool own = rl >= 1 && rl <= rows_here;
                    const int blo = own ? (int)kMagicBits : trash_bits;
                    const int bhi = own ? max_bits : trash_bits;
                    const float ncma = cmt[rl * p.units_per_row + uca];
                    const float ncmb = cmt[rl * p.units_per_row + ucb];
                    float e[VEC];
                    if (VEC == 4) {
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
                                             make_float2(ncc[VEC > 2 ? 2 : 0], ncc[VEC > 3 ? 3 : 0]));
                        }
                        float2 e01 = __fmul2_rn(c01, make_float2(gg[j].x, gg[j].y));
                        float2 e23 = __fmul2_rn(c23, make_float2(gg[j].z, gg[j].w));
                        if (MG && ((rr[j].x | rr[j].y) & (~mg.vmask << 16 | (~mg.vmask & 0xFFFFu)))) {
                            // words of a higher gain stage: that stage's pedestal
                            // and gain, no common mode; beyond the maps, 0
                            float ev[4] = {e01.x, e01.y, e23.x, e23.y};
                            const uint32_t wv[4] = {rr[j].x & 0xFFFFu, rr[j].x >> 16,
                                                    rr[j].y & 0xFFFFu, rr[j].y >> 16};
                            const size_t px = mod_base + (size_t)r * p.cols + (size_t)col;
#pragma unroll
                            for (int i = 0; i < 4; i++) {
                                const uint32_t st = wv[i] >> mg.shift;
                                if (st == 0) continue;
                                if (st >= mg.n_gains) {
                                    ev[i] = 0.0f;
                                    continue;
                                }
                                const size_t at = (size_t)st * p.frame_px + px + i;
                                ev[i] = __fmul_rn(
                                    __fsub_rn(__uint2float_rn(wv[i] & mg.vmask), mg.ped[at]),
                                    mg.inv_gain[at]);
                            }
                            e01 = make_float2(ev[0], ev[1]);
                            e23 = make_float2(ev[2], ev[3]);
                        }
                        e[0] = e01.x;
                        e[1] = e01.y;
                        e[2] = e23.x;
                        e[3] = e23.y;
                        // summary histogram of e (packed: bins of two pixels at once)
                        const float2 iw = make_float2(p.hist_inv_w, p.hist_inv_w);
                        const float2 nl = make_float2(p.hist_neg_lo_s, p.hist_neg_lo_s);
                        const float2 mg = make_float2(kMagic, kMagic);
                        const float2 u01 = __fadd2_rd(__ffma2_rn(e01, iw, nl), mg);
                        const float2 u23 = __fadd2_rd(__ffma2_rn(e23, iw, nl), mg);
                        atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u01.x), blo), bhi) - kMagicBits], 1u);
                        atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u01.y), blo), bhi) - kMagicBits], 1u);
                        atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u23.x), blo), bhi) - kMagicBits], 1u);
                        atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u23.y), blo), bhi) - kMagicBits], 1u);
                    } else {
                        float c0 = __fadd_rn(__fadd_rn(__uint2float_rn(r1[j]), p1[j]), ncma);
                        if (STACKED) c0 = __fadd_rn(__fadd_rn(c0, crt[rl]), ncc[0]);
                        e[0] = __fmul_rn(c0, g1[j]);
                        const float u = __fadd_rd(__fmaf_rn(e[0], p.hist_inv_w, p.hist_neg_lo_s),
                                                  kMagic);
                        atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u), blo), bhi) - kMagicBits], 1u);
                    }
                    float sv[VEC];
                    uint32_t seeds = 0;  // bit i: pixel i passes the seed threshold
#pragma unroll
                    for (int i = 0; i < VEC; i++) {
                        sv[i] = e[i] > p.zero_thr ? e[i] : 0.0f;
                        seeds |= (uint32_t)(sv[i] > p.seed_thr) << i;
                    }
                    if (VEC == 4)
                        *reinterpret_cast<float4*>(srow) = make_float4(sv[0], sv[1], sv[2], sv[3]);
                    else
                        srow[0] = sv[0];
                    if (own && out.corrected) {
                        const uint32_t off = (uint32_t)r * p.cols + (uint32_t)col;
                        float* dst = out.corrected + (size_t)f * p.frame_px + mod_base + off;
                        if (VEC == 4)
                            *reinterpret_cast<float4*>(dst) = make_float4(e[0], e[1], e[2], e[3]);
                        else
                            dst[0] = e[0];
                    }
                    // (a chunk's pixels share one word: col % 4 == 0 when VEC == 4)
                    if (own && seeds) atomicOr(&sbits[rl * WPR + (col >> 5)], seeds << (col & 31));
                }
            }
        }
        // the next tile's common mode, in flight during compaction and seeds
        if (t + step < n_tiles && tid < ncmt) cmv = tile_cm((uint32_t)(t + step), tid);

        __syncthreads();

        // compaction of the candidates: one bitmap word per thread, a warp
        // scan and one shared atomic per warp reserve each thread's slots
        // (list order is free); the words are cleared for the next tile
        const uint32_t n_words = (uint32_t)rows_here * WPR;
        for (uint32_t base = 0; base < n_words; base += nthr) {
            const uint32_t q = base + tid;
            uint32_t word = 0, rc = 0;  // rc: row << 16 | first column of the word
            if (q < n_words) {
                const uint32_t rl = 1 + q / WPR, w = q - (rl - 1) * WPR;
                word = sbits[rl * WPR + w];
                if (word) sbits[rl * WPR + w] = 0;
                rc = rl << 16 | 32 * w;
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
            if (lane == wl && tot) at0 = atomicAdd(&s_list_n, tot);
            at0 = __shfl_sync(wm, at0, wl);
            uint32_t at = at0 + incl - cnt;
            while (word && at < kSeedCap) {
                const int b = __ffs(word) - 1;
                word &= word - 1;
                list[at++] = rc + (uint32_t)b;
            }
        }
        __syncthreads();

        // 2. seeds: local maximum test, sums, count, centroid, emission
        const uint32_t n_list = s_list_n;
        const bool scan = n_list > kSeedCap;  // overflow: test every owned pixel
        const uint32_t n_work = scan ? (uint32_t)rows_here * (uint32_t)C : n_list;
        for (uint32_t base = 0; base < n_work; base += nthr) {
            const uint32_t j = base + tid;
            bool emit = false;
            pd_hit h;
            uint32_t n = 0, pix = 0;
            if (j < n_work) {
                int rl, c;
                if (scan) {
                    rl = 1 + (int)(j / (uint32_t)C);
                    c = (int)(j % (uint32_t)C);
                } else {
                    const uint32_t e = list[j];
                    rl = (int)(e >> 16);
                    c = (int)(e & 0xFFFFu);
                }
                const float* sc = stile + rl * P + 4 + c;
                const float sp = sc[0];
                if (sp > p.seed_thr) {
                    const float nb[9] = {sc[-(int)P - 1], sc[-(int)P], sc[-(int)P + 1],
                                         sc[-1],          sp,          sc[1],
                                         sc[P - 1],       sc[P],       sc[P + 1]};
                    const bool seed = sp > nb[0] && sp > nb[1] && sp > nb[2] && sp > nb[3] &&
                                      sp >= nb[5] && sp >= nb[6] && sp >= nb[7] && sp >= nb[8];
                    if (seed) {
                        float E = 0.0f, Mx = 0.0f, My = 0.0f;
                        uint32_t npix = 0;
#pragma unroll
                        for (int k = 0; k < 9; k++) {
                            const float ox = (float)(k % 3 - 1), oy = (float)(k / 3 - 1);
                            E = __fadd_rn(E, nb[k]);
                            Mx = __fadd_rn(Mx, __fmul_rn(nb[k], ox));
                            My = __fadd_rn(My, __fmul_rn(nb[k], oy));
                            npix += nb[k] > 0.0f;
                        }
                        atomicAdd(&hhit[summary_bin(E, p.hist_inv_w, p.hist_neg_lo_s, max_bits)],
                                  1u);
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
                            const int r = r0 - 1 + rl;
                            if (r == 0 || c == 0 || r == R - 1 || c == C - 1) flags |= PD_HIT_EDGE;
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
                const int leader = __ffs(mask) - 1;
                uint32_t slot = 0;
                if (lane == leader) slot = atomicAdd(out.n_hits, __popc(mask));
                slot = __shfl_sync(0xffffffffu, slot, leader);
                if (emit) {
                    slot += __popc(mask & ((1u << lane) - 1u));
                    atomicAdd(&p.count_map[pix], n);
                    if (slot < out.hit_capacity) out.hits[slot] = h;
                }
            }
        }
        __syncthreads();
        if (prefetcher && t + 2 * step < n_tiles) {
            TileWalk nx = walk;
            nx.next();
            nx.next();
            prefetch_tile_rows(raw, nx, bc.rb, p.rows, p.cols, p.frame_px);
        }
    }
    for (uint32_t b = tid; b < p.hist_bins; b += nthr) {
        if (hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)hpix[b]);
        if (hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)hhit[b]);
    }
}

template <int VEC, bool STACKED, bool MG = false>
__global__ void __launch_bounds__(kBandThreads, 2)
    stencil_band_kernel(ChainParams p, const uint16_t* __restrict__ raw,
                        uint32_t frame_base, CallOut out, BandConfig bc,
                        unsigned long long n_tiles, MultiGain mg) {
    extern __shared__ __align__(16) uint32_t band_smem[];
    __shared__ BandShared bsh;
    stencil_band_run<VEC, STACKED, MG, true>(p, raw, frame_base, out, bc, blockIdx.x, n_tiles,
                                             gridDim.x, band_smem, bsh, mg);
}

// ---------------------------------------------------------------------------
// Batched launches: the common mode of every (item, frame, unit) task of a
// batch of contexts in one persistent kernel, and every band tile of every
// item in one persistent stencil kernel.  Each CTA dispatches on the item's
// kind to the same device functions the single-context kernels use.
__device__ __forceinline__ uint32_t find_item(const BatchItem* items, uint32_t n_items,
                                              unsigned long long t, bool stencil) {
    uint32_t lo = 0, hi = n_items;  // last item whose first task <= t
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        const unsigned long long first = stencil ? items[mid].st_first : items[mid].cm_first;
        if (first <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// ALL_KINDS false: every item's common mode is a bank with pairs of
// pixels (kind 0) or rows (kind 4), the usual mix; the kernel then carries
// only those two paths (fewer registers).
template <bool ALL_KINDS>
__global__ void __launch_bounds__(512, 2)
    batch_cm_kernel(const BatchItem* __restrict__ items, uint32_t n_items,
                    unsigned long long n_tasks) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ CmBigShared big;
    __shared__ generic_cm::Shared gen;
    __shared__ RowWarpShared rows[16];
    for (unsigned long long t = blockIdx.x; t < n_tasks; t += gridDim.x) {
        const uint32_t i = find_item(items, n_items, t, false);
        const BatchItem& it = items[i];
        const uint32_t local = (uint32_t)(t - it.cm_first);
        if (it.cm_kind == 4) {  // 16 row units per task, one per warp
            const unsigned long long unit = (unsigned long long)local * 16 + (threadIdx.x >> 5);
            const unsigned long long units = (unsigned long long)it.n_frames * it.p.units_per_frame;
            if (unit < units) cm_rows_unit(it.p, it.raw, it.out.cm, unit, it.rows_magic, rows[threadIdx.x >> 5]);
            __syncthreads();
            continue;
        }
        if (!ALL_KINDS) {
            cm_big_unit<2>(it.p, it.raw, it.out.cm, it.cm_cfg, local, smem, big);
        } else {
            switch (it.cm_kind) {
                case 0: cm_big_unit<2>(it.p, it.raw, it.out.cm, it.cm_cfg, local, smem, big); break;
                case 1: cm_big_unit<1>(it.p, it.raw, it.out.cm, it.cm_cfg, local, smem, big); break;
                case 2: generic_cm::unit<true>(it.p, it.raw, it.out.cm, local, smem, gen); break;
                default: generic_cm::unit<false>(it.p, it.raw, it.out.cm, local, smem, gen); break;
            }
        }
        __syncthreads();  // shared memory is reused by the next task
    }
}

// VEC 4 or 1: every item uses that width; 0: each item its own.
template <int VEC>
__global__ void __launch_bounds__(kBandThreads, 2)
    batch_stencil_kernel(const BatchItem* __restrict__ items, uint32_t n_items) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ BandShared bsh;
    // the current item in shared memory: its parameters are read from there
    // rather than held in registers
    __shared__ __align__(16) BatchItem s_item;
    const unsigned long long G = gridDim.x, b = blockIdx.x;
    for (uint32_t i = 0; i < n_items; i++) {
        __syncthreads();  // the previous item is no longer read
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(items + i);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&s_item);
            for (uint32_t k = threadIdx.x; k < sizeof(BatchItem) / 4; k += blockDim.x)
                dst[k] = src[k];
        }
        __syncthreads();
        const BatchItem& it = s_item;
        const unsigned long long n = it.st_tiles;
        const unsigned long long first = (b + G - it.st_first % G) % G;
        if (first >= n) continue;
        if (VEC == 4 || (VEC == 0 && it.band_vec == 4))
            stencil_band_run<4>(it.p, it.raw, it.frame_base, it.out, it.band_cfg, first, n, G,
                                smem, bsh);
        else
            stencil_band_run<1>(it.p, it.raw, it.frame_base, it.out, it.band_cfg, first, n, G,
                                smem, bsh);
        __syncthreads();  // the next item re-zeroes the shared tile and histograms
    }
}

}  // namespace

cudaError_t launch_batch(const BatchItem* items_dev, uint32_t n_items,
                         unsigned long long cm_tasks, size_t cm_smem, size_t band_smem,
                         cudaStream_t stream, bool all_kinds, int vec) {
    int dev = 0;
    cudaGetDevice(&dev);
    static int attr_dev = -1;
    if (attr_dev != dev) {
        for (auto k : {batch_cm_kernel<true>, batch_cm_kernel<false>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kCmBigMaxSmem);
            if (e != cudaSuccess) return e;
        }
        for (auto k : {batch_stencil_kernel<0>, batch_stencil_kernel<4>, batch_stencil_kernel<1>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 200 * 1024);
            if (e != cudaSuccess) return e;
        }
        attr_dev = dev;
    }
    if (!items_dev) return cudaSuccess;  // attribute set-up only
    const unsigned sms = (unsigned)device_sm_count();
    if (cm_tasks) {
        unsigned long long grid = 2ull * sms;
        if (grid > cm_tasks) grid = cm_tasks;
        if (all_kinds)
            batch_cm_kernel<true><<<(unsigned)grid, 512, cm_smem, stream>>>(items_dev, n_items,
                                                                             cm_tasks);
        else
            batch_cm_kernel<false><<<(unsigned)grid, 512, cm_smem, stream>>>(items_dev, n_items,
                                                                              cm_tasks);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int per_sm = (int)((200 * 1024) / std::max<size_t>(band_smem, 1));
    per_sm = std::max(1, std::min(per_sm, 2));
    const unsigned grid_st = sms * (unsigned)per_sm;
    if (vec == 4)
        batch_stencil_kernel<4><<<grid_st, kBandThreads, band_smem, stream>>>(items_dev, n_items);
    else if (vec == 1)
        batch_stencil_kernel<1><<<grid_st, kBandThreads, band_smem, stream>>>(items_dev, n_items);
    else
        batch_stencil_kernel<0><<<grid_st, kBandThreads, band_smem, stream>>>(items_dev, n_items);
    return cudaGetLastError();
}

// 1.5 * 2^23 - w0 for the window base w0 = min(cut - 256, -128) (an integer)
float cm_rows_magic(const ChainParams& p) {
    return (float)(12582912.0 - std::min((double)p.cm_cut - 256.0, -128.0));
}

bool cm_rows_supported(const ChainParams& p) {
    const double lo = (double)p.cm_cut - 256.0;
    return p.unit_rows * p.unit_cols <= (uint32_t)kRowMaxPx && p.cm_cut > -1e6f &&
           p.cm_cut < 1e6f && lo == (double)(long long)lo;
}

cudaError_t launch_cm_rows(const ChainParams& p, const uint16_t* raw, uint32_t n_frames,
                           float* cm, cudaStream_t stream) {
    const unsigned long long items = (unsigned long long)n_frames * p.units_per_frame;
    if (items == 0) return cudaSuccess;
    // floor(d - w0) by a rounded-down fma with a magic addend
    const float magic_1 = cm_rows_magic(p);
    const unsigned long long blocks = (items + kRowWarps - 1) / kRowWarps;
    // units of up to 384 pixels (ASIC rows) hold 12 pixels a lane
    if (p.unit_px <= 384)
        cm_rows_kernel<12><<<(unsigned)blocks, 32 * kRowWarps, 0, stream>>>(p, raw, cm, items, magic_1);
    else
        cm_rows_kernel<kRowPerLane><<<(unsigned)blocks, 32 * kRowWarps, 0, stream>>>(p, raw, cm, items,
                                                                                  magic_1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
bool cm_big_supported(const ChainParams& p, const CmBigConfig& cfg) {
    return cfg.ok && p.unit_rows * p.unit_cols >= kCmBigMinPx &&
           cm_big_smem_bytes(p) <= kCmBigMaxSmem;
}

size_t cm_big_smem_bytes(const ChainParams& p) {
    const size_t codes = ((size_t)p.unit_rows * p.unit_cols * 2 + 15) / 16 * 16;
    return (size_t)(kCmBins + 4) * 4 + (size_t)kCandCap * 4 + codes;
}

CmBigConfig make_cm_big_config(const ChainParams& p) {
    CmBigConfig cfg{};
    cfg.ok = false;
    // the window [cut - 512, cut) must have 8*(cut - 512) an integer, so the
    // rounded-down fma computes floor(8 * (d - lo)) exactly
    const double cut = p.cm_cut;
    const double lo8 = (cut - 512.0) * 8.0;
    if (!(cut > -1e6 && cut < 1e6) || lo8 != (double)(long long)lo8) return cfg;
    cfg.magic_w = (float)(12582912.0 - lo8);
    cfg.w_lo = (float)(cut - 512.0);
    if ((double)cfg.magic_w != 12582912.0 - lo8) return cfg;
    const bool vec2 = p.unit_cols % 2 == 0 && p.cols % 2 == 0;
    cfg.vec = vec2 ? 2 : 1;
    const uint32_t tx = p.unit_cols / cfg.vec;
    if (tx == 0 || tx > 512) return cfg;
    cfg.tx = tx;
    cfg.ty = std::max<uint32_t>(1, 512 / tx);
    if (cfg.ty > p.unit_rows) cfg.ty = p.unit_rows;
    cfg.ok = true;
    return cfg;
}

static int g_attr_dev_cm = -1, g_attr_dev_band = -1;

cudaError_t launch_cm_big(const ChainParams& p, const CmBigConfig& cfg, const uint16_t* raw,
                          uint32_t n_frames, float* cm, cudaStream_t stream,
                          uint32_t stage_mask) {
    const unsigned long long items = (unsigned long long)n_frames * p.units_per_frame;
    if (items == 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_attr_dev_cm != dev) {
        for (auto k : {cm_big_kernel<2, false>, cm_big_kernel<1, false>, cm_big_kernel<2, true>,
                       cm_big_kernel<1, true>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kCmBigMaxSmem);
            if (e != cudaSuccess) return e;
        }
        g_attr_dev_cm = dev;
    }
    const size_t smem = cm_big_smem_bytes(p);
    const unsigned threads = cfg.tx * cfg.ty;
    auto k = cfg.vec == 2 ? (stage_mask ? cm_big_kernel<2, true> : cm_big_kernel<2, false>)
                          : (stage_mask ? cm_big_kernel<1, true> : cm_big_kernel<1, false>);
    k<<<(unsigned)items, threads, smem, stream>>>(p, raw, cm, cfg, stage_mask);
    return cudaGetLastError();
}

BandConfig make_band_config(const ChainParams& p) {
    BandConfig bc{};
    // a four-pixel chunk starts at a multiple of 4 and takes the common mode
    // of at most two units, which needs units at least two columns wide
    const bool vec4 = p.cols % 4 == 0 && p.module_px % 4 == 0 && p.frame_px % 4 == 0 &&
                      p.unit_cols >= 2;
    bc.vec = vec4 ? 4 : 1;
    bc.tx = p.cols / bc.vec;
    bc.ok = bc.tx <= kBandThreads;
    if (!bc.ok) return bc;
    bc.ty = std::max<uint32_t>(1, kBandThreads / bc.tx);
    bc.pitch = (p.cols + 8 + 3) / 4 * 4;  // 4 zero columns left, >= 1 right
    // about 12k pixels per band, at least 4 rows
    uint32_t rb = std::max<uint32_t>(4, 12288 / p.cols);
    rb = std::min<uint32_t>(rb, p.rows);
    // keep the shared memory of one CTA under about 100 KB
    while (rb > 1 && band_smem_bytes(p, rb, bc.pitch) > 100 * 1024) rb--;
    bc.rb = rb;
    bc.n_bands = (p.rows + rb - 1) / rb;
    return bc;
}

size_t band_smem_bytes(const ChainParams& p, uint32_t rb, uint32_t pitch) {
    return (size_t)(rb + 2) * pitch * 4 + (2 * (size_t)p.hist_bins + 4) * 4 +
           (size_t)kSeedCap * 4 + (size_t)(rb + 2) * p.units_per_row * 4 +
           (size_t)(rb + 2) * 4 +                           // row terms of the stacked mean
           (size_t)(rb + 1) * ((p.cols + 31) / 32) * 4;     // seed bitmap
}

cudaError_t launch_stencil_band(const ChainParams& p, const BandConfig& bc, const uint16_t* raw,
                                uint32_t n_frames, uint32_t frame_base, const CallOut& out,
                                cudaStream_t stream, const MultiGain* mg) {
    const unsigned long long n_tiles = (unsigned long long)n_frames * p.n_modules * bc.n_bands;
    if (n_tiles == 0) return cudaSuccess;
    if (mg && bc.vec != 4) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_attr_dev_band != dev) {
        for (auto k : {stencil_band_kernel<4, false>, stencil_band_kernel<1, false>,
                       stencil_band_kernel<4, true>, stencil_band_kernel<1, true>,
                       stencil_band_kernel<4, false, true>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 200 * 1024);
            if (e != cudaSuccess) return e;
        }
        g_attr_dev_band = dev;
    }
    const size_t smem = band_smem_bytes(p, bc.rb, bc.pitch);
    const unsigned threads = bc.tx * bc.ty;
    int per_sm = (int)((200 * 1024) / std::max<size_t>(smem, 1));
    per_sm = std::max(1, std::min(per_sm, 4));
    unsigned long long grid = (unsigned long long)device_sm_count() * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    const bool st = cm_kind(p) == PD_CM_MEAN_STACKED;
    const MultiGain m = mg ? *mg : MultiGain{};
    auto k = mg              ? stencil_band_kernel<4, false, true>
             : bc.vec == 4 && st ? stencil_band_kernel<4, true>
             : bc.vec == 4       ? stencil_band_kernel<4, false>
             : st                ? stencil_band_kernel<1, true>
                                 : stencil_band_kernel<1, false>;
    k<<<(unsigned)grid, threads, smem, stream>>>(p, raw, frame_base, out, bc, n_tiles, m);
    return cudaGetLastError();
}

}  // namespace pd
