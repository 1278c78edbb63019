// pd_lean.cu — the lean kernel pair of the chain.
//
//   cm_bank_kernel     common mode of one large unit per CTA (paper section
//                      "Common Mode", Fig. c; the estimator is the lower
//                      median over d < cut).  Pass A reads eight raw words per
//                      16-byte load (three rows in flight per thread) and
//                      turns them into histogram bins with 16-bit SIMD
//                      integer arithmetic (CodeMap in pd_lean.cuh): clamp,
//                      shift-add of the per-pixel offset, clamp; the codes
//                      stay in shared memory.  The bin of rank floor((n-1)/2)
//                      is found by a scan; pass B finds that bin's pixels
//                      among the thread's own codes (eight per 16-byte read,
//                      one shared atomic per warp to reserve their slots) and
//                      an exact selection over their binary32 d gives the
//                      median.  A median in the window's open bottom bin, or
//                      more candidates than the buffer holds, selects over
//                      the whole unit instead (same result).
//   stencil_lean_kernel dark, common mode, gain (Fig. b), the pixel
//                      histogram, zeroing, 3x3 local maximum, charge sum,
//                      count (Fig. e), centroid (Fig. f), hits and summaries
//                      for bands of full-width rows of a module; persistent
//                      over band tiles.  Each thread owns one four-pixel
//                      column chunk of the band and walks its rows; the
//                      corrected energies e of the band and its halo rows go
//                      to shared memory as they are, and only pixels with
//                      e above the seed threshold become candidates (a
//                      register bit per row, then a shared list).  The
//                      zeroing s = e > zero_thr ? e : 0 is applied where the
//                      3x3 sums read the neighbourhood.
//
// All arithmetic on values that reach an output is round-to-nearest in the
// chain's order (compiled with --fmad=false), as in pd_fast.cu.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "pd_dev.cuh"
#include "pd_lean.cuh"

namespace pd {

namespace {

// ---------------------------------------------------------------------------
// Bulk copies and mbarriers (inline PTX).
constexpr uint32_t kCopyWaitLimit = 1u << 20;  // try_wait rounds before giving up

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}
// orders this thread's generic-proxy shared-memory accesses before later
// asynchronous-proxy ones (a tensor copy into the same memory)
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// bounded wait for phase `parity` of the mbarrier; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint32_t limit = kCopyWaitLimit) {
    const uint32_t a = saddr(bar);
    for (uint32_t it = 0; it < limit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// 16-bit SIMD min / max of two lanes per word (sm_90 and later)
__device__ __forceinline__ uint32_t vmin_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t vmax_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// biased bin codes of two raw words: clamp(8 min(x, cap) + k, lo, hi) per lane
// (8 cap + k < 2^16 in each lane, so the shift-add carries nothing across)
__device__ __forceinline__ uint32_t code2(uint32_t x, uint32_t k, uint32_t cap2, uint32_t lo2,
                                          uint32_t hi2) {
    const uint32_t xm = vmin_u16x2(x, cap2);
    return vmin_u16x2(vmax_u16x2((xm << 3) + k, lo2), hi2);
}

// ---------------------------------------------------------------------------
// Common mode of one large unit, integer-coded.
struct BankShared {
    uint64_t bar;
    uint32_t gsum[kCmBins / 32];
    uint32_t swarp[32];
    uint32_t s_bin, s_rank, s_n, s_cand, s_prefix, s_rrank;
};

constexpr int kBankThreads = 512;
constexpr uint32_t kThreadGroups = 8;  // groups with a winning-bin code per thread (pass B)

// Block-wide location of rank k = target_of(total) in hist[0 .. PER * 512):
// each of the 512 threads sums PER bins, warp scans and the sixteen warp
// totals give every thread its prefix, and the thread whose bins hold rank k
// finds the bin.  *s_total, *s_bin (PER * 512 when no bin holds k) and
// *s_rank (rank within the bin).  All threads must call it.
template <int PER, class TargetFn>
__device__ __forceinline__ void rank_in_bins(const uint32_t* hist, TargetFn target_of,
                                             uint32_t* swarp, uint32_t* s_total, uint32_t* s_bin,
                                             uint32_t* s_rank) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t v[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; j++) {
        v[j] = hist[PER * tid + j];
        sum += v[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += x;
    }
    if (lane == 31) swarp[warp] = incl;
    if (tid == 0) *s_bin = PER * kBankThreads;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (uint32_t w = 0; w < kBankThreads / 32; w++) {
        const uint32_t t = swarp[w];
        before += w < warp ? t : 0u;
        total += t;
    }
    const uint32_t k = target_of(total);
    uint32_t lo = before + incl - sum;
    if (k < total && lo <= k && k < lo + sum) {
#pragma unroll
        for (int j = 0; j < PER; j++) {
            if (k < lo + v[j]) {
                *s_bin = PER * tid + j;
                *s_rank = k - lo;
                break;
            }
            lo += v[j];
        }
    }
    if (tid == 0) *s_total = total;
    __syncthreads();
}

// Exact element of rank `brank` among the mc binary32 values cand[0..mc)
// that all lie in the histogram bin [lo_b, lo_b + 1/8): 1024 sub-bins of
// 1/8192 ADU (d - lo_b rounded to nearest is monotone in d, so sub-bins stay
// ordered), then the few values of the target sub-bin are ranked by
// counting.  sub: 1024 words; scratch: mc words; few: up to mc floats.
// Thread 0 .. writes the result to *out.  All threads must call it.
__device__ void select_in_bin(const float* cand, uint32_t mc, float lo_b, uint32_t brank,
                              uint32_t* sub, uint32_t* scratch, float* few, uint32_t* swarp,
                              uint32_t* s_prefix, uint32_t* s_bin, uint32_t* s_rank,
                              uint32_t* s_nf, float* out) {
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    for (uint32_t i = tid; i < 1024 / 4; i += nthr)
        reinterpret_cast<uint4*>(sub)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) *s_nf = 0;
    __syncthreads();
    for (uint32_t t = tid; t < mc; t += nthr) {
        const float x = __fmul_rn(__fsub_rn(cand[t], lo_b), 8192.0f);
        const uint32_t sb = min((uint32_t)max(__float2int_rd(x), 0), 1023u);
        scratch[t] = sb;
        atomicAdd(&sub[sb], 1u);
    }
    __syncthreads();
    rank_in_bins<1024 / kBankThreads>(
        sub, [brank](uint32_t) { return brank; }, swarp, s_prefix, s_bin, s_rank);
    const uint32_t sbin = *s_bin, srank = *s_rank;
    for (uint32_t t = tid; t < mc; t += nthr)
        if (scratch[t] == sbin) few[atomicAdd(s_nf, 1u)] = cand[t];
    __syncthreads();
    const uint32_t nf = *s_nf;
    for (uint32_t t = tid; t < nf; t += nthr) {
        const uint32_t kt = order_key(few[t]);
        uint32_t less = 0, leq = 0;
        for (uint32_t j = 0; j < nf; j++) {
            const uint32_t kj = order_key(few[j]);
            less += kj < kt;
            leq += kj <= kt;
        }
        if (less <= srank && srank < leq) *out = few[t];
    }
}

// Pass A on one group of eight words: biased codes back to the group and one
// histogram increment per word (hb[code'] is hist[code' - bias]).
__device__ __forceinline__ void bank_codes(uint4* g, const uint4& k, uint32_t cap2, uint32_t lo2,
                                           uint32_t hi2, uint32_t* hb) {
    const uint4 x = *g;
    const uint4 y = make_uint4(code2(x.x, k.x, cap2, lo2, hi2), code2(x.y, k.y, cap2, lo2, hi2),
                               code2(x.z, k.z, cap2, lo2, hi2), code2(x.w, k.w, cap2, lo2, hi2));
    atomicAdd(hb + (y.x & 0xFFFFu), 1u);
    atomicAdd(hb + (y.x >> 16), 1u);
    atomicAdd(hb + (y.y & 0xFFFFu), 1u);
    atomicAdd(hb + (y.y >> 16), 1u);
    atomicAdd(hb + (y.z & 0xFFFFu), 1u);
    atomicAdd(hb + (y.z >> 16), 1u);
    atomicAdd(hb + (y.w & 0xFFFFu), 1u);
    atomicAdd(hb + (y.w >> 16), 1u);
    *g = y;
}

// 4-D tiled bulk tensor copy global -> shared (box at coordinates c0..c3 of
// the tensor map), counted against the mbarrier's transaction bytes
__device__ __forceinline__ void tensor_copy_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                               int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(saddr(bar))
        : "memory");
}

// The frames as the tensor [frame][period][group][8 words]: a period is
// cmap.t consecutive rows (t * cols a multiple of 8 words), a group 16 bytes.
// Unit u's rows of phase phi (global row = phi mod t) lie in one box of
// cmap.bp periods x cmap.w8 groups from (group g_lo(phi), period q_lo); the
// unit's staged buffer holds the t boxes one after the other, each padded to
// cmap.ne_box groups (a multiple of 8, so every box starts 128-byte aligned).
// The shared-memory regions of one bank item.
struct BankSmem {
    uint4* stage;    // t * ne_box groups of 8 words
    uint32_t* hist;  // kCmBins + 4 (spare at kCmBins)
    float* cand;     // candidate capacity
    uint32_t* cidx;  // candidate capacity
};

// Global first row and first column of item `it`'s unit, and its frame.
__device__ __forceinline__ void bank_unit_of(const ChainParams& p, uint32_t it, uint32_t* R0,
                                             uint32_t* c0, uint32_t* f) {
    *f = it / p.units_per_frame;
    const uint32_t u = it - *f * p.units_per_frame;
    const uint32_t m = u / p.units_per_module, um = u - m * p.units_per_module;
    *R0 = m * p.rows + (um / p.units_per_row) * p.unit_rows;
    *c0 = (um % p.units_per_row) * p.unit_cols;
}

// One tensor copy per row phase of item `it` into the stage (thread 0).
__device__ __forceinline__ void bank_issue(const ChainParams& p, const CodeMap& cmap,
                                           const CUtensorMap* frames, uint4* stage, uint64_t* bar,
                                           uint32_t it) {
    uint32_t R0, c0, f;
    bank_unit_of(p, it, &R0, &c0, &f);
    mbar_expect_tx(bar, cmap.t * cmap.bp * cmap.w8 * 16u);
    for (uint32_t ph = 0; ph < cmap.t; ph++)
        tensor_copy_4d(stage + ph * cmap.ne_box, frames, 0, (int)((ph * p.cols + c0) >> 3),
                       (int)(R0 / cmap.t), (int)f, bar);
}

// One bank item whose copy has been issued (its completion is phase `parity`
// of sh.bar); the histogram must be zero on entry and is zero again on
// return.  issue_next() runs on thread 0 once the stage is read (the next
// item's copy may start then).  False if the copy wait gave up.
template <class NextFn>
__device__ __forceinline__ bool cm_bank_item(const ChainParams& p, float* __restrict__ cm_out,
                                             const CmBigConfig& cfg, const CodeMap& cmap,
                                             const uint16_t* __restrict__ raw, uint32_t item,
                                             uint32_t parity, const BankSmem& sm,
                                             uint32_t cand_cap, BankShared& sh,
                                             uint32_t* __restrict__ err, NextFn issue_next) {
    uint4* stage = sm.stage;
    uint32_t* hist = sm.hist;
    float* cand = sm.cand;
    uint32_t* cidx = sm.cidx;
    const uint32_t W8 = cmap.w8, T = cmap.t;
    const uint32_t ne = T * cmap.ne_box;
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    const uint32_t cap2 = cmap.rcap * 0x10001u;
    const uint32_t lo2 = cmap.bias * 0x10001u;
    const uint32_t hi2 = (cmap.bias + kCmBins) * 0x10001u;
    uint32_t* hb = hist - cmap.bias;  // hb[code'] is hist[code' - bias]
    {
        uint32_t R0, c0, f;
        bank_unit_of(p, item, &R0, &c0, &f);
        const uint32_t u = item - f * p.units_per_frame;
        const uint32_t q_lo = R0 / T;
        const uint16_t* fr = raw + (size_t)f * p.frame_px;
        // the first per-pixel offsets K' of pass A (from the unit's map in
        // the staged layout) are loaded while the copies land
        const uint4* km = cmap.kmap + (size_t)u * ne;
        const uint4 zero4 = make_uint4(0, 0, 0, 0);
        uint4 k0 = tid < ne ? __ldg(km + tid) : zero4;
        uint4 k1 = tid + kBankThreads < ne ? __ldg(km + tid + kBankThreads) : zero4;
        uint4 k2 = tid + 2 * kBankThreads < ne ? __ldg(km + tid + 2 * kBankThreads) : zero4;
        // one thread waits for the copies; the others wait at the barrier
        // (which orders the copied data before their reads)
        const bool ok = tid != 0 ||
                        mbar_wait(&sh.bar, parity, cmap.wait_polls ? cmap.wait_polls : kCopyWaitLimit);
        if (__syncthreads_or(!ok)) {
            // the copies did not complete in time: report, give them a second
            // bounded wait (they write this CTA's shared memory), stop
            if (tid == 0) {
                atomicOr(err, 1u);
                mbar_wait(&sh.bar, parity);
            }
            return false;
        }

        // 1. pass A over the staged groups, three groups per round, the next
        //    round's offsets in flight
        for (uint32_t e = tid; e < ne; e += 3 * kBankThreads) {
            const uint32_t e3 = e + 3 * kBankThreads;
            const uint4 n0 = e3 < ne ? __ldg(km + e3) : zero4;
            const uint4 n1 = e3 + kBankThreads < ne ? __ldg(km + e3 + kBankThreads) : zero4;
            const uint4 n2 = e3 + 2 * kBankThreads < ne ? __ldg(km + e3 + 2 * kBankThreads) : zero4;
            bank_codes(stage + e, k0, cap2, lo2, hi2, hb);
            if (e + kBankThreads < ne) bank_codes(stage + e + kBankThreads, k1, cap2, lo2, hi2, hb);
            if (e + 2 * kBankThreads < ne)
                bank_codes(stage + e + 2 * kBankThreads, k2, cap2, lo2, hi2, hb);
            k0 = n0;
            k1 = n1;
            k2 = n2;
        }
        __syncthreads();

        // 2. the bin of rank floor((n-1)/2) among the values below the cut
        const uint32_t min_count = p.cm_min_count;
        rank_in_bins<kCmBins / kBankThreads>(
            hist,
            [min_count](uint32_t total) {
                return (total > 0 && total >= min_count) ? (total - 1) / 2 : total;
            },
            sh.swarp, &sh.s_n, &sh.s_bin, &sh.s_rank);
        const uint32_t n = sh.s_n;
        const uint32_t bin = sh.s_bin, brank = sh.s_rank;
        const bool none = n == 0 || n < min_count;
        // frame pixel of staged group e, word l
        auto staged_px = [&](uint32_t e, uint32_t l) -> uint32_t {
            const uint32_t ph = e / cmap.ne_box, g = e - ph * cmap.ne_box;
            const uint32_t pp = g / W8, k = g - pp * W8;
            return (q_lo + pp) * T * p.cols + 8 * (((ph * p.cols + c0) >> 3) + k) + l;
        };
        const uint32_t warp = tid >> 5;
        const uint32_t tgt = (bin + cmap.bias) * 0x10001u;
        uint32_t n_grp = 0;  // this thread's groups holding the winning bin
        if (!none && bin != 0) {
            // 3. pass B: the thread's groups that hold a code of the winning
            //    bin go to its own slots of the candidate buffer (no shared
            //    atomics, no warp coordination).  A halfword h of
            //    y = word ^ (target, target) is zero only if the word has a
            //    zero halfword when (y - 0x00010001) & ~y & 0x80008000 != 0
            //    (a borrow from a zero low half can flag the high half, but
            //    then the group matches anyway); the exact lanes are found
            //    after the barrier.
            uint16_t* slots = reinterpret_cast<uint16_t*>(cidx) + tid * kThreadGroups;
            for (uint32_t e = tid; e < ne; e += kBankThreads) {
                const uint4 v = stage[e];
                const uint32_t y0 = v.x ^ tgt, y1 = v.y ^ tgt, y2 = v.z ^ tgt, y3 = v.w ^ tgt;
                const uint32_t h = ((y0 - 0x00010001u) & ~y0) | ((y1 - 0x00010001u) & ~y1) |
                                   ((y2 - 0x00010001u) & ~y2) | ((y3 - 0x00010001u) & ~y3);
                if (h & 0x80008000u) {
                    if (n_grp < kThreadGroups) slots[n_grp] = (uint16_t)e;
                    n_grp++;
                }
            }
        }
        // exact matching pixels of the thread's groups, and a block scan of
        // their counts for the compact candidate array
        uint32_t n_px = 0;
        if (!none && bin != 0) {
            const uint16_t* slots = reinterpret_cast<const uint16_t*>(cidx) + tid * kThreadGroups;
            for (uint32_t i = 0; i < min(n_grp, kThreadGroups); i++) {
                const uint4 v = stage[slots[i]];
                const uint32_t w[4] = {v.x ^ tgt, v.y ^ tgt, v.z ^ tgt, v.w ^ tgt};
#pragma unroll
                for (int j = 0; j < 4; j++)
                    n_px += ((w[j] & 0xFFFFu) == 0) + ((w[j] >> 16) == 0);
            }
        }
        uint32_t incl = n_px;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += x;
        }
        const bool ovf = n_grp > kThreadGroups;
        if (lane == 31) sh.swarp[warp] = incl;
        if (tid == 0) sh.s_cand = 0;
        __syncthreads();
        if (ovf) sh.s_cand = 1;  // a thread's slots overflowed
        uint32_t before = incl - n_px, mc = 0;
        for (uint32_t w = 0; w < kBankThreads / 32; w++) {
            const uint32_t c = sh.swarp[w];
            before += w < warp ? c : 0u;
            mc += c;
        }
        // 4. the staged position of each matching pixel at its place in a
        //    compact list (in the histogram's words, free now), then one
        //    thread per candidate loads its raw word and pedestal
        uint32_t* qlist = hist;
        if (!none && bin != 0 && mc <= cand_cap) {
            const uint16_t* slots = reinterpret_cast<const uint16_t*>(cidx) + tid * kThreadGroups;
            uint32_t at = before;
            for (uint32_t i = 0; i < min(n_grp, kThreadGroups); i++) {
                const uint32_t e = slots[i];
                const uint4 v = stage[e];
                const uint32_t w[4] = {v.x ^ tgt, v.y ^ tgt, v.z ^ tgt, v.w ^ tgt};
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (((w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu) == 0) qlist[at++] = e * 8 + j;
            }
        }
        __syncthreads();  // the stage is no longer read
        if (!none && bin != 0 && mc <= cand_cap) {
            const float* npf = p.nped;
            for (uint32_t t = tid; t < mc; t += kBankThreads) {
                const uint32_t q = qlist[t];
                const uint32_t px = staged_px(q >> 3, q & 7u);
                cand[t] = __fadd_rn(__uint2float_rn(fr[px]), npf[px]);
            }
        }
        __syncthreads();
        // the next item's copies (after the candidates' loads, which would
        // otherwise queue behind them) land while this item is ranked
        if (tid == 0) issue_next();
        const bool over = sh.s_cand != 0 || mc > cand_cap;
        if (none) {
            if (tid == 0) cm_out[item] = 0.0f;
        } else if (bin != 0 && !over) {
            // the exact rank inside the bin
            const float lo_b = __fadd_rn(cfg.w_lo, __fmul_rn((float)bin, 0.125f));
            select_in_bin(cand, mc, lo_b, brank, hist, cidx, reinterpret_cast<float*>(hist + 1024),
                          sh.swarp, &sh.s_prefix, &sh.s_bin, &sh.s_rank, &sh.s_rrank,
                          cm_out + item);
        } else {
            // whole-unit exact selection (bottom bin or candidate overflow)
            const uint32_t P0 = R0 * p.cols + c0;
            const float* npf = p.nped;
            auto unit_key = [&](uint32_t i) -> uint32_t {
                const uint32_t px = P0 + (i / p.unit_cols) * p.cols + i % p.unit_cols;
                const float d = __fadd_rn(__uint2float_rn(fr[px]), npf[px]);
                return d < p.cm_cut ? order_key(d) : kSent;
            };
            const uint32_t key = block_radix_select(unit_key, p.unit_px, (n - 1) / 2, hist,
                                                    &sh.s_prefix, &sh.s_rrank);
            if (tid == 0) cm_out[item] = key_value(key);
        }
        __syncthreads();  // the histogram and candidates are no longer read
        for (uint32_t i = tid; i < (kCmBins + 4) / 4; i += kBankThreads)
            reinterpret_cast<uint4*>(hist)[i] = make_uint4(0, 0, 0, 0);
        if (tid == 0) sh.s_cand = 0;
        __syncthreads();
    }
    return true;
}

// Persistent: CTA b takes items b, b + grid, ...; the next item's copies are
// issued as soon as pass B has finished reading the stage, so they land
// while the current item's candidates are ranked.
__global__ void __launch_bounds__(kBankThreads, 2)
    cm_bank_kernel(ChainParams p, float* __restrict__ cm_out, CmBigConfig cfg, CodeMap cmap,
                   const __grid_constant__ CUtensorMap frames, const uint16_t* __restrict__ raw,
                   uint32_t n_items, uint32_t* __restrict__ err) {
    extern __shared__ __align__(128) uint4 stage[];  // t * ne_box groups of 8 words
    __shared__ BankShared sh;
    const uint32_t ne = cmap.t * cmap.ne_box;
    BankSmem sm;
    sm.stage = stage;
    sm.hist = reinterpret_cast<uint32_t*>(stage + ne);
    sm.cand = reinterpret_cast<float*>(sm.hist + kCmBins + 4);
    sm.cidx = reinterpret_cast<uint32_t*>(sm.cand + kCandCap);
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&sh.bar, 1);
        fence_mbar_init();
        if (blockIdx.x < n_items) bank_issue(p, cmap, &frames, stage, &sh.bar, blockIdx.x);
    }
    for (uint32_t i = tid; i < (kCmBins + 4) / 4; i += kBankThreads)
        reinterpret_cast<uint4*>(sm.hist)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) sh.s_cand = 0;
    __syncthreads();  // mbarrier initialised, histogram zero

    uint32_t parity = 0;
    for (uint32_t item = blockIdx.x; item < n_items; item += gridDim.x, parity ^= 1u) {
        const uint32_t next = item + gridDim.x;
        const bool ok = cm_bank_item(p, cm_out, cfg, cmap, raw, item, parity, sm, kCandCap, sh,
                                     err, [&] {
                                         if (next < n_items) {
                                             // order this item's generic stage accesses
                                             // before the copy
                                             fence_async_smem();
                                             bank_issue(p, cmap, &frames, stage, &sh.bar, next);
                                         }
                                     });
        if (!ok) return;
    }
}

// ---------------------------------------------------------------------------
// Lean stencil over bands of full-width rows.
constexpr uint32_t kLeanThreads = 512;

struct LeanRow {
    uint2 rw;   // four raw words
    float4 np;  // their negated pedestals
    float4 g;   // their inverse gains
};

// Shared memory of the lean stencil: the staged raw rows (STAGE), the tile
// of corrected energies, the two summary histograms, the candidate list,
// the common mode per tile row (not COLBANK), the list counters and the
// stage's mbarrier.
struct LeanSmem {
    const uint16_t* stg;
    float* tile;       // (rb + 2) x pitch
    uint32_t* hpix;    // hist_bins
    uint32_t* hhit;    // hist_bins
    uint32_t* list;    // list_cap
    float* cmt;        // (rb + 2) x units_per_row
    uint32_t* list_n;  // 2
    uint64_t* stage_bar;
};

// A thread's fixed part in every tile: its four-pixel chunk (column col of
// chunk column cx), its row lane ty, the common-mode units of its chunk, and
// the seed threshold's histogram bin; computed once per kernel.
struct LeanLane {
    uint32_t cx, ty;
    int col;
    uint32_t uca, ucb;  // units of the chunk's first and last pixel
    int split;          // pixels i >= split take unit ucb
    int seed_bin;       // every e > seed_thr has a bin >= seed_bin
    int n_own_full;     // own rows of a full band
};

__device__ __forceinline__ LeanLane lean_lane(const ChainParams& p, const LeanConfig& lc) {
    LeanLane L;
    const uint32_t tid = threadIdx.x;
    L.cx = tid % lc.tx;
    L.ty = tid / lc.tx;
    L.col = 4 * (int)L.cx;
    L.uca = (uint32_t)L.col / p.unit_cols;
    L.ucb = (uint32_t)(L.col + 3) / p.unit_cols;
    L.split = (int)(L.ucb * p.unit_cols) - L.col;
    L.seed_bin = (int)summary_bin(p.seed_thr, p.hist_inv_w, p.hist_neg_lo_s,
                                  (int)(kMagicBits + p.hist_bins - 1));
    L.n_own_full = lc.rb > L.ty ? ((int)lc.rb - 1 - (int)L.ty) / (int)lc.ty + 1 : 0;
    return L;
}

// One tile (band `band` of module m of frame f, list counter `par`).  The
// tile's pad columns must be zero and list_n[par] zero on entry.  Threads
// with rowlane false own no rows (blocks larger than tx * ty).
// issue_next() runs on thread 0 once the stage is read.  False if a staged
// copy's wait gave up.  ONEUNIT (per-row table only): every four-pixel chunk
// lies inside one common-mode unit (unit_cols a multiple of 4).
template <bool COLBANK, bool CORR, bool STAGE, bool ONEUNIT, class NextFn>
__device__ __forceinline__ bool lean_tile(const ChainParams& p, const uint16_t* __restrict__ raw,
                                          uint32_t frame_base, const CallOut& out,
                                          const LeanConfig& lc, const LeanSmem& sm,
                                          const LeanLane& L, uint32_t f, uint32_t m, uint32_t band,
                                          uint32_t par, bool rowlane, uint32_t* __restrict__ err,
                                          NextFn issue_next) {
    const uint32_t P = lc.pitch, RB = lc.rb;
    const uint16_t* stg = sm.stg;
    float* tile = sm.tile;
    uint32_t* hpix = sm.hpix;
    uint32_t* hhit = sm.hhit;
    uint32_t* list = sm.list;
    float* cmt = sm.cmt;
    uint32_t* list_n = sm.list_n;
    uint64_t* stage_bar = sm.stage_bar;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t TY = lc.ty;
    const uint32_t ty = L.ty;
    const int R = (int)p.rows, C = (int)p.cols;
    const int col = L.col;
    const uint32_t uca = L.uca, ucb = L.ucb;
    const int split = L.split;
    const int last_bin = (int)p.hist_bins - 1;
    const float2 iw2 = make_float2(p.hist_inv_w, p.hist_inv_w);
    const float2 nl2 = make_float2(p.hist_neg_lo_s, p.hist_neg_lo_s);
    const float2 mg2 = make_float2(kMagic, kMagic);
    // rows holding a histogram bin >= seed_bin are scanned for candidates
    const int seed_bin = L.seed_bin;
    const uint32_t T = STAGE ? lc.stage_t : 1u;
    const int n_own_full = L.n_own_full;
    {
        const int r0 = (int)band * (int)RB;
        const int rows_here = min((int)RB, R - r0);
        const size_t mod_base = (size_t)m * p.module_px;
        const uint16_t* fr = raw + (size_t)f * p.frame_px + mod_base;
        const float* npm = p.nped + mod_base;
        const float* gm = p.inv_gain + mod_base;
        const float* cmf = out.cm + (size_t)f * p.units_per_frame + (size_t)m * p.units_per_module;
        // stage row of module row r: r + srow0
        const int srow0 =
            STAGE ? (int)(m * p.rows) - (((int)(m * p.rows) + r0 - 1) & ~(int)(T - 1)) : 0;
        const uint32_t soff = (uint32_t)srow0 * p.cols;  // stage word of frame word off: off + soff
        // the chunk's two common-mode values (COLBANK), loaded before the
        // wait for the stage so that their latency overlaps it
        float ca = 0.0f, cb = 0.0f;
        if (COLBANK) {
            ca = -__ldcg(cmf + uca);
            cb = -__ldcg(cmf + ucb);
        }
        if (STAGE) {
            // one thread waits for the copy; the barrier orders its data
            // before every thread's reads
            const bool ok = tid != 0 ||
                            mbar_wait(stage_bar, par, lc.wait_polls ? lc.wait_polls : kCopyWaitLimit);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(err, 2u);
                    mbar_wait(stage_bar, par);  // the copy still writes this CTA's memory
                }
                return false;
            }
        }

        // negated common mode of the chunk's pixels (COLBANK), or of every
        // (tile row, unit column) in shared memory
        float2 n01 = make_float2(0.0f, 0.0f), n23 = n01;
        if (COLBANK) {
            const float a = ca, b = cb;
            n01 = make_float2(split > 0 ? a : b, split > 1 ? a : b);
            n23 = make_float2(split > 2 ? a : b, split > 3 ? a : b);
        } else {
            // (entry i: tile row i / upr, unit column i % upr; the divisions
            // are skipped for one unit per row and for one-row units)
            const uint32_t upr = p.units_per_row;
            for (uint32_t i = tid; i < (uint32_t)(rows_here + 2) * upr; i += nthr) {
                const uint32_t ri = upr == 1 ? i : i / upr;
                const int r = r0 - 1 + (int)ri;
                const uint32_t ur = p.unit_rows == 1 ? (uint32_t)r : (uint32_t)r / p.unit_rows;
                cmt[i] = r >= 0 && r < R ? -__ldcg(cmf + ur * upr + (i - ri * upr)) : 0.0f;
            }
            __syncthreads();
        }

        // e of four pixels of module row r, from a row of loads
        auto correct = [&](const LeanRow& x, int rl, float2& e01, float2& e23) {
            const float2 d01 = __fadd2_rn(raw_pair(x.rw.x), make_float2(x.np.x, x.np.y));
            const float2 d23 = __fadd2_rn(raw_pair(x.rw.y), make_float2(x.np.z, x.np.w));
            float2 m01 = n01, m23 = n23;
            if (!COLBANK && ONEUNIT) {
                const float a = cmt[rl * p.units_per_row + uca];
                m01 = make_float2(a, a);
                m23 = m01;
            } else if (!COLBANK) {
                const float a = cmt[rl * p.units_per_row + uca];
                const float b = cmt[rl * p.units_per_row + ucb];
                m01 = make_float2(split > 0 ? a : b, split > 1 ? a : b);
                m23 = make_float2(split > 2 ? a : b, split > 3 ? a : b);
            }
            e01 = __fmul2_rn(__fadd2_rn(d01, m01), make_float2(x.g.x, x.g.y));
            e23 = __fmul2_rn(__fadd2_rn(d23, m23), make_float2(x.g.z, x.g.w));
        };
        auto load = [&](int r) -> LeanRow {
            const uint32_t off = (uint32_t)r * p.cols + (uint32_t)col;
            LeanRow x;
            if (STAGE)
                x.rw = *reinterpret_cast<const uint2*>(stg + off + soff);
            else
                x.rw = __ldg(reinterpret_cast<const uint2*>(fr + off));
            x.np = __ldg(reinterpret_cast<const float4*>(npm + off));
            x.g = __ldg(reinterpret_cast<const float4*>(gm + off));
            return x;
        };

        // 1. halo rows (tile rows 0 and rows_here + 1): e only, zero outside
        //    the module; done by the last two row lanes, which own the
        //    fewest rows
        auto halo = [&](int rl) {
            const int r = r0 - 1 + rl;
            float4 ev = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (r >= 0 && r < R) {
                float2 e01, e23;
                correct(load(r), rl, e01, e23);
                ev = make_float4(e01.x, e01.y, e23.x, e23.y);
            }
            *reinterpret_cast<float4*>(tile + rl * P + 4 + col) = ev;
        };
        if (TY == 1) {
            halo(0);
            halo(rows_here + 1);
        } else if (ty == TY - 1) {
            halo(0);
        } else if (ty == TY - 2) {
            halo(rows_here + 1);
        }

        // 2. own rows r0 + ty + i TY (tile row 1 + ty + i TY): e to the tile,
        //    the pixel histogram, a bit per row whose largest bin reaches the
        //    seed threshold's; rows are processed in pairs from two register
        //    sets, so the next row's loads are in flight while a row is
        //    processed
        const int n_own = !rowlane               ? 0
                          : rows_here == (int)RB ? n_own_full
                          : rows_here > (int)ty  ? (rows_here - 1 - (int)ty) / (int)TY + 1
                                                 : 0;
        uint32_t cmask = 0;  // bit i: own row i may hold a candidate
        auto own_row = [&](const LeanRow& x, int i) {
            const int rl = 1 + (int)ty + i * (int)TY;
            float2 e01, e23;
            correct(x, rl, e01, e23);
            const float2 u01 = __fadd2_rd(__ffma2_rn(e01, iw2, nl2), mg2);
            const float2 u23 = __fadd2_rd(__ffma2_rn(e23, iw2, nl2), mg2);
            const int b0 = min(__viaddmax_s32(__float_as_int(u01.x), -(int)kMagicBits, 0), last_bin);
            const int b1 = min(__viaddmax_s32(__float_as_int(u01.y), -(int)kMagicBits, 0), last_bin);
            const int b2 = min(__viaddmax_s32(__float_as_int(u23.x), -(int)kMagicBits, 0), last_bin);
            const int b3 = min(__viaddmax_s32(__float_as_int(u23.y), -(int)kMagicBits, 0), last_bin);
            atomicAdd(&hpix[b0], 1u);
            atomicAdd(&hpix[b1], 1u);
            atomicAdd(&hpix[b2], 1u);
            atomicAdd(&hpix[b3], 1u);
            *reinterpret_cast<float4*>(tile + rl * P + 4 + col) =
                make_float4(e01.x, e01.y, e23.x, e23.y);
            if (CORR) {
                float* dst = out.corrected + (size_t)f * p.frame_px + mod_base +
                             (size_t)(r0 + rl - 1) * p.cols + col;
                *reinterpret_cast<float4*>(dst) = make_float4(e01.x, e01.y, e23.x, e23.y);
            }
            if (max(__vimax3_s32(b0, b1, b2), b3) >= seed_bin) cmask |= 1u << i;
        };
        if (n_own > 0) {
            const int rs = (int)TY;  // rows between a thread's own rows
            LeanRow a = load(r0 + (int)ty), b;
            for (int i = 0; i < n_own; i += 2) {
                if (i + 1 < n_own) b = load(r0 + (int)ty + (i + 1) * rs);
                own_row(a, i);
                if (i + 1 >= n_own) break;
                if (i + 2 < n_own) a = load(r0 + (int)ty + (i + 2) * rs);
                own_row(b, i + 1);
            }
        }
        // candidate pixels (e > seed_thr) of the marked rows into the tile's
        // list, one reservation per thread (rare: the thread reads its own
        // rows back from the tile)
        if (cmask) {
            auto bits4 = [&](int i) -> uint32_t {
                const int rl = 1 + (int)ty + i * (int)TY;
                const float4 ev = *reinterpret_cast<const float4*>(tile + rl * P + 4 + col);
                return (uint32_t)(ev.x > p.seed_thr) | (uint32_t)(ev.y > p.seed_thr) << 1 |
                       (uint32_t)(ev.z > p.seed_thr) << 2 | (uint32_t)(ev.w > p.seed_thr) << 3;
            };
            uint32_t n_px = 0;
            for (uint32_t mm = cmask; mm; mm &= mm - 1) n_px += __popc(bits4(__ffs(mm) - 1));
            if (n_px) {
                uint32_t at = atomicAdd(&list_n[par], n_px);
                for (uint32_t mm = cmask; mm; mm &= mm - 1) {
                    const int i = __ffs(mm) - 1;
                    const uint32_t rl = 1 + ty + (uint32_t)i * TY;
                    for (uint32_t bb = bits4(i); bb; bb &= bb - 1, at++)
                        if (at < lc.list_cap)
                            list[at] = rl << 16 | ((uint32_t)col + (uint32_t)(__ffs(bb) - 1));
                }
            }
        }
        __syncthreads();
        // the stage is read: the next tile's rows land during the seeds
        if (tid == 0) issue_next();

        // 3. seeds: local maximum on s = e > zero_thr ? e : 0 with the raster
        //    tie rule, 3x3 sums, count, centroid, emission
        const uint32_t n_list = list_n[par];
        if (tid == 0) list_n[par ^ 1u] = 0;  // the next tile's counter (read last tile)
        const bool scan = n_list > lc.list_cap;  // overflow: test every own pixel
        const uint32_t n_work = scan ? (uint32_t)rows_here * (uint32_t)C : n_list;
        const float z = p.zero_thr;
        for (uint32_t base = 0; base < n_work; base += nthr) {
            if (base + (tid & ~31u) >= n_work) break;  // the whole warp is past the list
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
                const float* sc = tile + rl * P + 4 + c;
                const float sp = sc[0];
                if (sp > p.seed_thr) {
                    float nb[9] = {sc[-(int)P - 1], sc[-(int)P], sc[-(int)P + 1],
                                   sc[-1],          sp,          sc[1],
                                   sc[P - 1],       sc[P],       sc[P + 1]};
#pragma unroll
                    for (int k = 0; k < 9; k++) nb[k] = nb[k] > z ? nb[k] : 0.0f;
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
                        atomicAdd(&hhit[summary_bin(E, p.hist_inv_w, p.hist_neg_lo_s,
                                                    (int)(kMagicBits + p.hist_bins - 1))],
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
                const int lane = tid & 31;
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
        __syncthreads();  // the tile is rewritten by the next band
    }
    return true;
}

// Tiles first, first + step, ... < n_tiles (tile t: band t % n_bands of module
// (t / n_bands) % n_modules of frame t / (n_bands n_modules)).  COLBANK: the
// common-mode units span the module's full height, so a thread's four pixels
// take the same two values on every row of a tile.  CORR: write corrected
// frames.  STAGE: the tile's raw rows come by one tensor copy (the frames as
// [frame][period][group][8 words]) into shared memory; the next tile's copy
// is issued once the rows are read and lands while the seeds are tested.
// ONEUNIT: as in lean_tile.
template <bool COLBANK, bool CORR, bool STAGE, bool ONEUNIT = false>
__global__ void __launch_bounds__(kLeanThreads, 2)
    stencil_lean_kernel(ChainParams p, const uint16_t* __restrict__ raw, uint32_t frame_base,
                        CallOut out, LeanConfig lc, unsigned long long n_tiles,
                        const __grid_constant__ CUtensorMap frames, uint32_t* __restrict__ err) {
    extern __shared__ __align__(128) float lean_smem[];
    __shared__ uint32_t list_n[2];
    __shared__ uint64_t stage_bar;
    const uint32_t P = lc.pitch, RB = lc.rb;
    // staged raw rows (STAGE), 128-byte aligned, then the float tile
    const uint32_t stage_words = STAGE ? lc.stage_bp * lc.stage_g * 8u : 0u;
    LeanSmem sm;
    sm.stg = reinterpret_cast<const uint16_t*>(lean_smem);
    sm.tile = lean_smem + ((stage_words / 2 + 31u) & ~31u);
    sm.hpix = reinterpret_cast<uint32_t*>(sm.tile + (RB + 2) * P);
    sm.hhit = sm.hpix + p.hist_bins;
    sm.list = sm.hhit + p.hist_bins;
    sm.cmt = reinterpret_cast<float*>(sm.list + lc.list_cap);
    sm.list_n = list_n;
    sm.stage_bar = &stage_bar;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;

    // the copy of tile tt's raw rows (thread 0): from the period holding the
    // row above the band (T is a power of two, so & ~(T - 1) floors to a
    // period, -1 included)
    auto issue = [&](unsigned long long tt) {
        const uint32_t T = lc.stage_t;
        const unsigned long long mb = tt / lc.n_bands;
        const uint32_t band = (uint32_t)(tt - mb * lc.n_bands);
        const uint32_t f = (uint32_t)(mb / p.n_modules);
        const uint32_t m = (uint32_t)(mb - (unsigned long long)f * p.n_modules);
        const int first = ((int)(m * p.rows + band * RB) - 1) & ~(int)(T - 1);
        mbar_expect_tx(&stage_bar, lc.stage_bp * lc.stage_g * 16u);
        tensor_copy_4d(lean_smem, &frames, 0, 0, first / (int)T, (int)f, &stage_bar);
    };
    if (STAGE && tid == 0) {
        mbar_init(&stage_bar, 1);
        fence_mbar_init();
        if (blockIdx.x < n_tiles) issue(blockIdx.x);
    }
    for (uint32_t i = tid; i < (RB + 2) * P; i += nthr) sm.tile[i] = 0.0f;
    for (uint32_t i = tid; i < 2 * p.hist_bins; i += nthr) sm.hpix[i] = 0;
    if (tid < 2) list_n[tid] = 0;
    __syncthreads();

    const LeanLane lane = lean_lane(p, lc);
    const unsigned long long first = blockIdx.x, step = gridDim.x;
    TileWalk walk(first, step, lc.n_bands, p.n_modules);
    // unstaged: the last thread (a halo lane, which owns the fewest rows)
    // asks L2 for the raw rows (halo rows included) of the tile after next
    // once a tile is done, so that their loads find them there
    const bool prefetcher = !STAGE && tid == nthr - 1;
    auto prefetch = [&](const TileWalk& w) {
        prefetch_tile_rows(raw, w, RB, p.rows, p.cols, p.frame_px);
    };
    if (prefetcher && first + step < n_tiles) {
        TileWalk nx = walk;
        nx.next();
        prefetch(nx);
    }
    uint32_t par = 0;
    for (unsigned long long t = first; t < n_tiles; t += step, walk.next(), par ^= 1u) {
        const bool ok = lean_tile<COLBANK, CORR, STAGE, ONEUNIT>(
            p, raw, frame_base, out, lc, sm, lane, walk.f, walk.m, walk.band, par, true, err, [&] {
                if (STAGE && t + step < n_tiles) {
                    fence_async_smem();  // order the generic reads of the stage before the copy
                    issue(t + step);
                }
            });
        if (!ok) return;
        if (prefetcher && t + 2 * step < n_tiles) {
            TileWalk nx = walk;
            nx.next();
            nx.next();
            prefetch(nx);
        }
    }
    for (uint32_t b = tid; b < p.hist_bins; b += nthr) {
        if (sm.hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)sm.hpix[b]);
        if (sm.hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)sm.hhit[b]);
    }
}

// ---------------------------------------------------------------------------
// The lean pair as one persistent launch over a work queue.  Items are
// claimed in order from a global counter; superstep s holds the bank items
// of frames [sK, sK + K) and then the stencil tiles of frames
// [(s-1)K, sK), so a tile's raw rows were read by its bank items one
// superstep earlier (K frames of raw, a few tens of MB, stay in L2) and no
// kernel boundary separates the two kinds.  A tile waits (bounded) until
// both banks of its module have published their common mode.  A tile only
// waits on items earlier in the queue, and a CTA only ever waits on such
// items while it holds a later one, so the waits cannot form a cycle
// whichever CTAs are resident.

struct QueuePlan {
    uint32_t n_frames, K;     // frames of the launch, frames per superstep
    uint32_t U, TPF;          // bank items and tiles per frame
    uint32_t n_items;         // n_frames (U + TPF)
};

constexpr uint32_t kDepWaitLimit = 1u << 22;  // polls of a tile's dependency

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* a) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// First queue index of superstep s.
__device__ __forceinline__ uint32_t queue_start(const QueuePlan& q, uint32_t s) {
    const uint32_t cm_frames = min(s * q.K, q.n_frames);
    const uint32_t st_frames = s ? min((s - 1) * q.K, q.n_frames) : 0u;
    return cm_frames * q.U + st_frames * q.TPF;
}

// Queue index i as a bank item (*cm true, *item) or a tile (*cm false, tile
// index *item = f * TPF + m * n_bands + band).
__device__ __forceinline__ void queue_decode(const QueuePlan& q, uint32_t i, bool* cm,
                                             uint32_t* item) {
    const uint32_t first = min(q.K, q.n_frames) * q.U;
    uint32_t s = i < first ? 0u : 1u + (i - first) / (q.K * (q.U + q.TPF));
    while (s > 0 && queue_start(q, s) > i) s--;
    while (queue_start(q, s + 1) <= i) s++;
    const uint32_t j = i - queue_start(q, s);
    const uint32_t cm_here = s * q.K < q.n_frames ? min(q.K, q.n_frames - s * q.K) * q.U : 0u;
    *cm = j < cm_here;
    *item = *cm ? s * q.K * q.U + j : (s - 1) * q.K * q.TPF + (j - cm_here);
}

__global__ void __launch_bounds__(kBankThreads, 2)
    chain_queue_kernel(ChainParams p, const uint16_t* __restrict__ raw, uint32_t frame_base,
                       CallOut out, CmBigConfig cfg, CodeMap cmap, LeanConfig lc, QueuePlan q,
                       const __grid_constant__ CUtensorMap frames, uint32_t* __restrict__ qsync,
                       uint32_t* __restrict__ err) {
    extern __shared__ __align__(128) uint4 qsmem[];
    __shared__ BankShared sh;
    __shared__ uint32_t list_n[2];
    __shared__ uint32_t s_kind, s_item;  // the claimed item, decoded by thread 0
    const uint32_t tid = threadIdx.x;
    uint32_t* counter = qsync;  // the queue
    uint32_t* done = qsync + 1;  // per (frame, module): banks published
    // bank item view of the shared memory
    BankSmem bs;
    bs.stage = qsmem;
    bs.hist = reinterpret_cast<uint32_t*>(qsmem + cmap.t * cmap.ne_box);
    bs.cand = reinterpret_cast<float*>(bs.hist + kCmBins + 4);
    bs.cidx = reinterpret_cast<uint32_t*>(bs.cand + kCandCap);
    // tile view of the same memory (the summary histograms are flushed to
    // global memory before a bank item reuses it)
    LeanSmem ts;
    ts.stg = nullptr;
    ts.tile = reinterpret_cast<float*>(qsmem);
    ts.hpix = reinterpret_cast<uint32_t*>(ts.tile + (lc.rb + 2) * lc.pitch);
    ts.hhit = ts.hpix + p.hist_bins;
    ts.list = ts.hhit + p.hist_bins;
    ts.cmt = nullptr;
    ts.list_n = list_n;
    ts.stage_bar = nullptr;
    const bool rowlane = tid < lc.tx * lc.ty;
    const LeanLane lane = lean_lane(p, lc);

    // thread 0 decodes a claimed index for the block (kind 2: past the end)
    auto publish = [&](uint32_t i) {
        bool cm = false;
        uint32_t it = 0;
        if (i < q.n_items) queue_decode(q, i, &cm, &it);
        s_kind = i >= q.n_items ? 2u : cm ? 0u : 1u;
        s_item = it;
    };
    if (tid == 0) {
        mbar_init(&sh.bar, 1);
        fence_mbar_init();
        publish(atomicAdd(counter, 1u));
    }
    __syncthreads();
    uint32_t parity = 0, par = 0;
    int prev = -1;             // kind of the previous item: 0 bank, 1 tile
    bool staged = false;       // thread 0: this bank item's copy was issued
    auto flush_hists = [&] {
        for (uint32_t b = tid; b < p.hist_bins; b += blockDim.x) {
            if (ts.hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)ts.hpix[b]);
            if (ts.hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)ts.hhit[b]);
        }
    };
    while (true) {
        const uint32_t kind = s_kind, item = s_item;
        if (kind == 2) break;
        uint32_t nxt = 0;
        if (tid == 0) nxt = atomicAdd(counter, 1u);  // claimed now, read at the item's end
        if (kind == 0) {
            if (prev == 1) {
                flush_hists();
                __syncthreads();  // the histograms are read before the bank item overwrites them
            }
            if (tid == 0 && !staged) {
                fence_async_smem();  // the tile's generic accesses before the copy
                bank_issue(p, cmap, &frames, bs.stage, &sh.bar, item);
            }
            if (prev != 0) {
                for (uint32_t k = tid; k < (kCmBins + 4) / 4; k += blockDim.x)
                    reinterpret_cast<uint4*>(bs.hist)[k] = make_uint4(0, 0, 0, 0);
                if (tid == 0) sh.s_cand = 0;
                // (the item's first barrier orders these stores before its passes)
            }
            bool next_staged = false;
            const bool ok = cm_bank_item(p, out.cm, cfg, cmap, raw, item, parity, bs, kCandCap, sh,
                                         err, [&] {
                                             if (nxt >= q.n_items) return;
                                             bool ncm;
                                             uint32_t nitem;
                                             queue_decode(q, nxt, &ncm, &nitem);
                                             if (ncm) {
                                                 fence_async_smem();
                                                 bank_issue(p, cmap, &frames, bs.stage, &sh.bar,
                                                            nitem);
                                                 next_staged = true;
                                             }
                                         });
            parity ^= 1u;
            if (!ok) return;
            staged = next_staged;
            // publish the bank's common mode: every thread's stores (the
            // winning thread's included) are fenced before the count
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                const uint32_t f = item / p.units_per_frame;
                const uint32_t m = (item - f * p.units_per_frame) / p.units_per_module;
                atomicAdd(done + f * p.n_modules + m, 1u);
            }
            prev = 0;
        } else {
            const uint32_t f = item / q.TPF;
            const uint32_t rem = item - f * q.TPF;
            const uint32_t m = rem / lc.n_bands, band = rem - m * lc.n_bands;
            if (prev != 1) {
                // zero summaries, zero pad columns, fresh list counters
                for (uint32_t k = tid; k < 2 * p.hist_bins; k += blockDim.x) ts.hpix[k] = 0;
                for (uint32_t k = tid; k < (lc.rb + 2) * 8; k += blockDim.x) {
                    const uint32_t r = k >> 3, c = k & 7u;
                    ts.tile[r * lc.pitch + (c < 4 ? c : p.cols + c)] = 0.0f;
                }
                if (tid < 2) list_n[tid] = 0;
                par = 0;
            }
            // both banks of the module have published their common mode
            bool ok = true;
            if (tid == 0) {
                const uint32_t* d = done + f * p.n_modules + m;
                const uint32_t limit = lc.wait_polls ? lc.wait_polls : kDepWaitLimit;
                uint32_t it = 0;
                while (ld_acquire_gpu(d) < p.units_per_module && ++it < limit) __nanosleep(64);
                ok = it < limit;
                if (!ok) atomicOr(err, 4u);
            }
            if (__syncthreads_or(!ok)) return;
            lean_tile<true, false, false, false>(p, raw, frame_base, out, lc, ts, lane, f, m, band, par,
                                          rowlane, err, [] {});
            par ^= 1u;
            prev = 1;
        }
        if (tid == 0) publish(nxt);
        __syncthreads();
    }
    if (prev == 1) flush_hists();
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side of the integer codes.
namespace {

// floor(a + b) of two doubles, exactly (TwoSum keeps the rounding error)
long long floor_sum(double a, double b) {
    const double s = a + b;
    const double bb = s - a;
    const double err = (a - (s - bb)) + (b - bb);
    const double fs = std::floor(s);
    if (s == fs) return (long long)fs - (err < 0.0 ? 1 : 0);
    return (long long)fs;
}

}  // namespace

bool build_code_map(const ChainParams& p, const float* pedestal, std::vector<uint16_t>* kmap,
                    CodeMap* out) {
    if (p.frame_px % 8) return false;
    if (!(p.cm_cut > -1e6f && p.cm_cut < 1e6f)) return false;
    // periods of t rows whose length is a multiple of 8 words tile the frame
    uint32_t gcd = 8;
    while (p.cols % gcd) gcd >>= 1;
    const uint32_t T = 8 / gcd;
    if (((size_t)p.n_modules * p.rows) % T) return false;
    const double cut = p.cm_cut;
    const double lo = cut - 512.0;
    const double D = std::max(std::fabs(lo), std::fabs(cut));
    const size_t fpx = p.frame_px;
    long long fmin = 0, fmax = 0, rcap = 0;
    std::vector<int32_t> F(fpx);
    for (size_t i = 0; i < fpx; i++) {
        const float ped = pedestal[i];
        if (!std::isfinite(ped)) return false;
        if (ped != 0.0f) {
            // d = x - ped is exact in binary32 while |d| < 2^24 ulp-units of ped
            int ex = 0;
            std::frexp((double)ped, &ex);  // |ped| in [2^(ex-1), 2^ex)
            const int q = std::max(ex - 24, -149);
            if (!(D < std::ldexp(1.0, 24 + q))) return false;
        }
        const long long fv = floor_sum(-8.0 * (double)ped, -8.0 * lo);
        if (fv < -(1LL << 30) || fv > (1LL << 30)) return false;
        F[i] = (int32_t)fv;
        // raw words at or above ceil((4096 - F) / 8) are in the spare bin
        const long long need = 4096 - fv;
        const long long rc = need <= 0 ? 0 : (need + 7) / 8;
        fmin = i ? std::min(fmin, fv) : fv;
        fmax = i ? std::max(fmax, fv) : fv;
        rcap = i ? std::max(rcap, rc) : rc;
    }
    const long long bias = fmin < 0 ? -fmin : 0;
    const long long kmax = std::max(fmax + bias, bias + 4096);
    if (rcap > 65535 || 8 * rcap + kmax > 65535) return false;
    // box of a unit's rows of one phase: periods q_lo .. q_hi, groups
    // g_lo(phase) .. g_hi(phase) of a period
    auto unit_pos = [&](uint32_t u, uint32_t* R0, uint32_t* c0) {
        const uint32_t m = u / p.units_per_module, um = u % p.units_per_module;
        *R0 = m * p.rows + (um / p.units_per_row) * p.unit_rows;
        *c0 = (um % p.units_per_row) * p.unit_cols;
    };
    uint32_t w8 = 0, bp = 0;
    for (uint32_t u = 0; u < p.units_per_frame; u++) {
        uint32_t R0, c0;
        unit_pos(u, &R0, &c0);
        bp = std::max(bp, (R0 + p.unit_rows - 1) / T - R0 / T + 1);
        for (uint32_t ph = 0; ph < T; ph++)
            w8 = std::max(w8, (ph * p.cols + c0 + p.unit_cols - 1) / 8 - (ph * p.cols + c0) / 8 + 1);
    }
    if (w8 > 256 || bp > 256) return false;
    const uint32_t ne_box = (bp * w8 + 7) / 8 * 8;
    const size_t per_unit = (size_t)T * ne_box * 8;
    const uint16_t junk = (uint16_t)(bias + 4096);
    kmap->assign((size_t)p.units_per_frame * per_unit, junk);
    const size_t tpx = (size_t)T * p.cols;  // words per period
    for (uint32_t u = 0; u < p.units_per_frame; u++) {
        uint32_t R0, c0;
        unit_pos(u, &R0, &c0);
        const uint32_t q_lo = R0 / T;
        for (uint32_t ph = 0; ph < T; ph++) {
            uint16_t* dst = kmap->data() + (size_t)u * per_unit + (size_t)ph * ne_box * 8;
            const uint32_t g_lo = (ph * p.cols + c0) / 8;
            for (uint32_t pp = 0; pp < bp; pp++)
                for (uint32_t k = 0; k < w8; k++)
                    for (uint32_t l = 0; l < 8; l++) {
                        const size_t ppx = 8 * ((size_t)g_lo + k) + l;  // word of the period
                        if (ppx >= tpx) continue;
                        const uint32_t rp = (uint32_t)(ppx / p.cols);
                        const uint32_t col = (uint32_t)(ppx % p.cols);
                        const size_t R = (size_t)(q_lo + pp) * T + rp;
                        if (rp != ph || R < R0 || R >= (size_t)R0 + p.unit_rows || col < c0 ||
                            col >= c0 + p.unit_cols)
                            continue;
                        dst[((size_t)pp * w8 + k) * 8 + l] = (uint16_t)(F[R * p.cols + col] + bias);
                    }
        }
    }
    *out = CodeMap{nullptr, w8, (uint32_t)bias, (uint32_t)rcap, T, bp, ne_box, 2};
    return true;
}

size_t cm_bank_smem_bytes(const ChainParams& p, const CodeMap& cmap) {
    (void)p;
    return (size_t)cmap.t * cmap.ne_box * 16 + (size_t)(kCmBins + 4) * 4 + (size_t)kCandCap * 8;
}

bool cm_bank_supported(const ChainParams& p, const CodeMap& cmap) {
    return p.unit_rows * p.unit_cols >= kCmBigMinPx && cm_bank_smem_bytes(p, cmap) <= 110 * 1024;
}

static int g_attr_dev_bank = -1;

// cuTensorMapEncodeTiled from the driver, looked up once
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// The call's frames as the tensor [frame][period][group][8 words] of uint16
// with the bank item's box.
static cudaError_t encode_bank_map(const ChainParams& p, const CodeMap& cmap,
                                   const uint16_t* raw, uint32_t n_frames, CUtensorMap* map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const uint64_t G = (uint64_t)cmap.t * p.cols / 8;
    const cuuint64_t dims[4] = {8, G, (cuuint64_t)p.frame_px / ((cuuint64_t)cmap.t * p.cols),
                                n_frames};
    const cuuint64_t strides[3] = {16, G * 16, (cuuint64_t)p.frame_px * 2};
    const cuuint32_t box[4] = {8, cmap.w8, cmap.bp, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<uint16_t*>(raw), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_cm_bank(const ChainParams& p, const CmBigConfig& cfg, const CodeMap& cmap,
                           const uint16_t* raw, uint32_t n_frames, float* cm, uint32_t* err,
                           cudaStream_t stream) {
    const unsigned long long items = (unsigned long long)n_frames * p.units_per_frame;
    if (items == 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_attr_dev_bank != dev) {
        cudaError_t e = cudaFuncSetAttribute(cm_bank_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             110 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(cm_bank_kernel,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        g_attr_dev_bank = dev;
    }
    CUtensorMap map;
    cudaError_t me = encode_bank_map(p, cmap, raw, n_frames, &map);
    if (me != cudaSuccess) return me;
    const size_t smem = cm_bank_smem_bytes(p, cmap);
    const unsigned long long grid = std::min<unsigned long long>(
        items, (unsigned long long)std::max<uint32_t>(cmap.ctas_per_sm, 1) * device_sm_count());
    cm_bank_kernel<<<(unsigned)grid, kBankThreads, smem, stream>>>(p, cm, cfg, cmap, map, raw,
                                                                   (uint32_t)items, err);
    return cudaGetLastError();
}

}  // namespace pd

// ---------------------------------------------------------------------------
// Host side of the lean stencil.
namespace pd {

constexpr size_t kLeanSmemTwo = 108 * 1024;  // two CTAs per SM
constexpr size_t kLeanSmemMax = 200 * 1024;

// periods the stage holds: the band's rows, the rows above and below it,
// and up to stage_t - 1 rows before them (the copy starts on a period)
void set_stage_periods(LeanConfig& lc) {
    if (lc.stage_t) lc.stage_bp = (lc.rb + 1 + 2 * lc.stage_t - 1) / lc.stage_t;
}
bool staged(const LeanConfig& lc) { return lc.stage_t != 0 && lc.stage_bp <= 256; }

LeanConfig make_lean_config(const ChainParams& p, uint32_t rb) {
    LeanConfig lc{};
    lc.ok = false;
    // four-pixel chunks start 8-byte aligned in every frame and module, and a
    // chunk takes the common mode of at most two units
    if (p.cols % 4 || p.module_px % 4 || p.frame_px % 4 || p.unit_cols < 2) return lc;
    if (p.cols / 4 > kLeanThreads || p.cols > 65535) return lc;
    if (cm_kind(p) == PD_CM_MEAN_STACKED || cm_after_gain(p)) return lc;
    lc.tx = p.cols / 4;
    lc.ty = std::max<uint32_t>(1, kLeanThreads / lc.tx);
    lc.pitch = p.cols + 8;
    lc.colbank = p.unit_rows == p.rows ? 1u : 0u;
    lc.list_cap = 4096;
    lc.stage_t = 0;  // the band height is chosen without the stage
    const bool dflt = rb == 0;
    if (dflt) {
        // the tallest band two CTAs per SM hold (at most 16 rows per row
        // lane), then split evenly over the module's rows
        LeanConfig t = lc;
        t.rb = 1;
        while (t.rb < p.rows && (t.rb + lc.ty) / lc.ty <= 16) {
            t.rb++;
            set_stage_periods(t);
            if (lean_smem_bytes(p, t) > kLeanSmemTwo) {
                t.rb--;
                break;
            }
        }
        const uint32_t nb = (p.rows + t.rb - 1) / t.rb;
        rb = (p.rows + nb - 1) / nb;
    }
    rb = std::min(rb, p.rows);
    // own rows per thread fit a 64-bit candidate mask (4 bits per row)
    while (rb > 1 && (rb + lc.ty - 1) / lc.ty > 16) rb--;
    lc.rb = rb;
    set_stage_periods(lc);
    // the default keeps two CTAs per SM; a requested height may take one
    const size_t limit = dflt ? kLeanSmemTwo : kLeanSmemMax;
    while (lc.rb > 1 && lean_smem_bytes(p, lc) > limit) {
        lc.rb--;
        set_stage_periods(lc);
    }
    lc.n_bands = (p.rows + lc.rb - 1) / lc.rb;
    lc.ok = lean_smem_bytes(p, lc) <= limit;
    // staged raw where it costs no band height: the fewest rows per period
    // whose words fill 16-byte groups (at most 256 groups, the tensor copy's
    // box limit), frames a whole number of periods and of 16-byte groups.
    // On the 2.2 Mpx sensor the stage would cut the band from 47 to 31 rows,
    // and the shorter bands' per-tile costs outweigh the faster rows
    // (measured 117.7 k against 122.1 k frames/s), so it stays off there.
    // (nor a CTA per SM: a band that fits two CTAs per SM unstaged keeps them)
    const size_t stage_limit = lean_smem_bytes(p, lc) <= kLeanSmemTwo ? kLeanSmemTwo : limit;
    for (uint32_t t = 1; t <= 8 && lc.ok; t *= 2)
        if ((t * p.cols) % 8 == 0) {
            if (t * p.cols / 8 <= 256 && (p.frame_px / p.cols) % t == 0 && p.frame_px % 8 == 0 &&
                encode_fn() != nullptr) {
                lc.stage_t = t;
                lc.stage_g = t * p.cols / 8;
                set_stage_periods(lc);
                if (!staged(lc) || lean_smem_bytes(p, lc) > stage_limit) lc.stage_t = 0;
            }
            break;
        }
    return lc;
}

size_t lean_smem_bytes(const ChainParams& p, const LeanConfig& lc) {
    const size_t stage = staged(lc) ? ((size_t)lc.stage_bp * lc.stage_g * 16 + 127) / 128 * 128 : 0;
    return stage + (size_t)(lc.rb + 2) * lc.pitch * 4 + 2 * (size_t)p.hist_bins * 4 +
           (size_t)lc.list_cap * 4 + (lc.colbank ? 0 : (size_t)(lc.rb + 2) * p.units_per_row * 4);
}

static int g_attr_dev_lean = -1;

namespace {
// the stencil instance for a common-mode layout: column banks, a per-row
// table, or a per-row table whose chunks each lie in one unit
template <bool CORR, bool STAGE>
auto lean_pick(bool colbank, bool oneunit) {
    return colbank   ? stencil_lean_kernel<true, CORR, STAGE, false>
           : oneunit ? stencil_lean_kernel<false, CORR, STAGE, true>
                     : stencil_lean_kernel<false, CORR, STAGE, false>;
}
}  // namespace

cudaError_t launch_stencil_lean(const ChainParams& p, const LeanConfig& lc, const uint16_t* raw,
                                uint32_t n_frames, uint32_t frame_base, const CallOut& out,
                                uint32_t* err, cudaStream_t stream) {
    const unsigned long long n_tiles = (unsigned long long)n_frames * p.n_modules * lc.n_bands;
    if (n_tiles == 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_attr_dev_lean != dev) {
        for (auto k : {stencil_lean_kernel<true, false, false>, stencil_lean_kernel<true, true, false>,
                       stencil_lean_kernel<false, false, false>, stencil_lean_kernel<false, true, false>,
                       stencil_lean_kernel<true, false, true>, stencil_lean_kernel<true, true, true>,
                       stencil_lean_kernel<false, false, true>, stencil_lean_kernel<false, true, true>,
                       stencil_lean_kernel<false, false, false, true>,
                       stencil_lean_kernel<false, true, false, true>,
                       stencil_lean_kernel<false, false, true, true>,
                       stencil_lean_kernel<false, true, true, true>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kLeanSmemMax);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (e != cudaSuccess) return e;
        }
        g_attr_dev_lean = dev;
    }
    const bool stage = staged(lc);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (stage) {
        // the call's frames as [frame][period][group][8 words] of uint16
        PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
        if (!enc || !err) return cudaErrorNotSupported;
        const uint64_t G = lc.stage_g;
        const cuuint64_t dims[4] = {8, G, (cuuint64_t)p.frame_px / ((cuuint64_t)lc.stage_t * p.cols),
                                    n_frames};
        const cuuint64_t strides[3] = {16, G * 16, (cuuint64_t)p.frame_px * 2};
        const cuuint32_t box[4] = {8, lc.stage_g, lc.stage_bp, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<uint16_t*>(raw), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const size_t smem = lean_smem_bytes(p, lc);
    const unsigned threads = lc.tx * lc.ty;
    const uint32_t per_sm = lc.ctas_per_sm ? lc.ctas_per_sm : (smem <= kLeanSmemTwo ? 2u : 1u);
    unsigned long long grid = (unsigned long long)device_sm_count() * per_sm;
    if (grid > n_tiles) grid = n_tiles;
    const bool corr = out.corrected != nullptr;
    // per-row tables with every four-pixel chunk inside one unit take one
    // table read per row
    const bool one = !lc.colbank && p.unit_cols % 4 == 0;
    auto k = stage ? (corr ? lean_pick<true, true>(lc.colbank, one)
                           : lean_pick<false, true>(lc.colbank, one))
                   : (corr ? lean_pick<true, false>(lc.colbank, one)
                           : lean_pick<false, false>(lc.colbank, one));
    k<<<(unsigned)grid, threads, smem, stream>>>(p, raw, frame_base, out, lc, n_tiles, map, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host side of the work-queue launch.

constexpr size_t kQueueSuperstepBytes = 20u << 20;  // raw per superstep (stays in L2)

size_t queue_smem_bytes(const ChainParams& p, const CodeMap& cmap, const LeanConfig& lc) {
    return std::max(cm_bank_smem_bytes(p, cmap), lean_smem_bytes(p, lc));
}

bool queue_supported(const ChainParams& p, const CodeMap& cmap, const LeanConfig& lc) {
    return lc.ok && lc.colbank && !staged(lc) && lc.tx * lc.ty <= kBankThreads &&
           cm_bank_supported(p, cmap) && queue_smem_bytes(p, cmap, lc) <= 110 * 1024 &&
           p.cols >= 8;
}

size_t queue_sync_words(const ChainParams& p, uint32_t n_frames) {
    return 1 + (size_t)n_frames * p.n_modules;
}

static int g_attr_dev_queue = -1;

cudaError_t launch_chain_queue(const ChainParams& p, const CmBigConfig& cfg, const CodeMap& cmap,
                               const LeanConfig& lc, const uint16_t* raw, uint32_t n_frames,
                               uint32_t frame_base, const CallOut& out, uint32_t* qsync,
                               uint32_t* err, cudaStream_t stream) {
    if (n_frames == 0) return cudaSuccess;
    const uint64_t per_frame = (uint64_t)p.units_per_frame + (uint64_t)p.n_modules * lc.n_bands;
    if ((uint64_t)n_frames * per_frame >= (1ull << 31)) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_attr_dev_queue != dev) {
        cudaError_t e = cudaFuncSetAttribute(chain_queue_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             110 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(chain_queue_kernel,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        g_attr_dev_queue = dev;
    }
    CUtensorMap map;
    cudaError_t e = encode_bank_map(p, cmap, raw, n_frames, &map);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(qsync, 0, queue_sync_words(p, n_frames) * 4, stream))) return e;
    QueuePlan q;
    q.n_frames = n_frames;
    q.K = (uint32_t)std::max<size_t>(1, kQueueSuperstepBytes / ((size_t)p.frame_px * 2));
    q.U = p.units_per_frame;
    q.TPF = p.n_modules * lc.n_bands;
    q.n_items = (uint32_t)(n_frames * per_frame);
    const size_t smem = queue_smem_bytes(p, cmap, lc);
    const unsigned grid = (unsigned)std::min<uint64_t>(q.n_items, 2ull * device_sm_count());
    chain_queue_kernel<<<grid, kBankThreads, smem, stream>>>(p, raw, frame_base, out, cfg, cmap,
                                                             lc, q, map, qsync, err);
    return cudaGetLastError();
}

}  // namespace pd
