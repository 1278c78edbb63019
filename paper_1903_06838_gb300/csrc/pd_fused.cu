// pd_fused.cu — the whole chain in one pass per module, for modules whose
// common-mode units are full-height column banks (the CSPAD layout: 185 x
// 388 sensors split into two 185 x 194 banks; paper section "Common Mode",
// Fig. c), or with common mode off.
//
// One CTA owns one (frame, module) at a time (persistent over all of them):
//
//   A. Dark subtraction d = raw + (-pedestal) (Fig. b) and a histogram of d
//      per bank over 3584 bins of 1/8 ADU whose window [cut - 448, cut) ends
//      at the cut; the low byte of every pixel's bin code stays in shared
//      memory (71 KB for a CSPAD sensor).
//   B. Exact lower median of d < cut per bank: the bin of rank
//      floor((n-1)/2) by a scan; the pixels whose code byte matches (the
//      bin's pixels plus aliases 32 ADU apart) are gathered, their d is
//      recomputed and filtered to the bin, and 1024 sub-bins of 1/8192 ADU
//      plus counting among the few values left give the median.  A median in
//      the open bottom bin, or too many candidates, falls back to a radix
//      select over the whole bank (same result).
//   C. Common mode, gain, zeroing, summary histogram of e, 3x3 local
//      maximum, charge sum, count, centroid, hits (Figs. b, e, f): a sweep
//      down the module in bands of 2*TY rows through a ring of 24 rows of
//      the zeroed signal s, so every row is computed once (no halo rows).
//      Seeds of a band's last row wait for the next band, which brings the
//      row below.  Seed candidates are compacted per warp into one of three
//      rotating lists, so a band needs a single barrier.
//
// Raw is read from DRAM once (pass A); pass C reads it again while the
// module's 143 KB are still in L2.  Bit-exact to the oracle: every value
// that reaches an output is computed with round-to-nearest operations in the
// chain's order (compiled with --fmad=false); bin codes use the exact
// floor-by-magic-number identities of pd_dev.cuh.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pd_dev.cuh"
#include "pd_fast.cuh"

// rows of loads a thread keeps in flight in pass A
#ifndef PD_FUSED_UNROLL
#define PD_FUSED_UNROLL 4
#endif

namespace pd {

namespace {

constexpr uint32_t kFuBins = kFusedCmBins;       // 1/8 ADU: window [cut - 448, cut)
constexpr uint32_t kFuHistWords = kFuBins + 4;   // + spare bin (d >= cut) + pad
constexpr uint32_t kFuPosCap = 4096;             // matching code bytes (incl. aliases)
constexpr uint32_t kFuCandCap = 2048;            // values in the median bins
constexpr uint32_t kFuRing = 24;                 // rows of the zeroed-signal ring
constexpr uint32_t kFuListCap = 1536;            // seed candidates per band (x3)
constexpr uint32_t kFuGroups = kFuBins / 32;     // 112 groups of 32 bins

struct FuShared {
    uint32_t gsum[kFusedMaxUnits][128];
    uint32_t swarp[32];
    uint32_t s_n[kFusedMaxUnits], s_bin[kFusedMaxUnits], s_rank[kFusedMaxUnits];
    uint32_t s_cand[kFusedMaxUnits];
    uint32_t s_pos, s_prefix, s_rrank, s_total, s_sbin, s_srank;
    uint32_t s_list[3];
    float s_cm[kFusedMaxUnits];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void red_shared_add1(uint32_t addr) {
    asm volatile("red.shared.add.u32 [%0], 1;\n" ::"r"(addr) : "memory");
}

// 0x80 in every byte of x that is zero, 0 elsewhere (exact, no carries
// between bytes).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
    return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
}

// Common-mode bin code (bit pattern kMagicBits + floor(8 (d - lo)), clipped
// to [kMagicBits, kMagicBits + kFuBins]) of one value.
__device__ __forceinline__ int fu_code(float d, float magic_w) {
    const int b = __float_as_int(__fmaf_rd(d, 8.0f, magic_w));
    return min(max(b, (int)kMagicBits), (int)(kMagicBits + kFuBins));
}

__device__ __forceinline__ float raw_at(const uint16_t* fr, uint32_t off) {
    return __uint2float_rn(fr[off]);
}

}  // namespace

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 2)
    chain_module_kernel(ChainParams p, FusedConfig fc, const uint16_t* __restrict__ raw,
                        uint32_t n_frames, uint32_t frame_base, CallOut out) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ FuShared sh;

    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t TX = fc.tx, TY = fc.ty, P = fc.pitch;
    const uint32_t tx = tid % TX, ty = tid / TX;
    const bool active = ty < TY;  // threads past TX * TY only join barriers and warp ops
    const int R = (int)p.rows, C = (int)p.cols;
    const uint32_t c4 = 4 * tx;
    const uint32_t U = p.units_per_row;
    const bool median = cm_kind(p) == PD_CM_MEDIAN;

    uint32_t* codes32 = smem;                                    // region A
    float* ring = reinterpret_cast<float*>(smem);                // region A (pass C)
    uint32_t* lists = smem + kFuRing * P;                        // 3 x kFuListCap
    uint32_t* regb = smem + fc.region_a_words;                   // region B
    uint32_t* pos = regb;                                        // kFuPosCap (pass B)
    float* cand = reinterpret_cast<float*>(regb + kFuPosCap);    // kFuCandCap
    uint32_t* sub = regb + kFuPosCap + kFuCandCap;               // 1024
    uint32_t* hpix = regb + fc.region_b_words;                   // hist_bins + 4
    uint32_t* hhit = hpix + p.hist_bins + 4;                     // hist_bins
    const uint32_t cap_u = kFuCandCap / kFusedMaxUnits;

    // unit and histogram address of each pixel of this thread's chunk: the
    // red at hb[i] + 4 * bits lands on bin bits - kMagicBits of the unit's
    // histogram (32-bit shared-window arithmetic, modulo 2^32)
    uint32_t unit_of[4];
    uint32_t hb[4];
    const uint32_t regb_addr = smem_addr(regb);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        unit_of[i] = median ? (c4 + i) / p.unit_cols : 0u;
        hb[i] = regb_addr + unit_of[i] * kFuHistWords * 4u - kMagicBits * 4u;
    }
    const int max_bits = (int)(kMagicBits + p.hist_bins - 1);
    const float2 iw = make_float2(p.hist_inv_w, p.hist_inv_w);
    const float2 nl = make_float2(p.hist_neg_lo_s, p.hist_neg_lo_s);
    const float2 mg = make_float2(kMagic, kMagic);

    for (uint32_t i = tid; i < 2 * p.hist_bins + 4; i += nthr) hpix[i] = 0;

    const unsigned long long n_items = (unsigned long long)n_frames * p.n_modules;
    for (unsigned long long item = blockIdx.x; item < n_items; item += gridDim.x) {
        const uint32_t f = (uint32_t)(item / p.n_modules);
        const uint32_t m = (uint32_t)(item % p.n_modules);
        const size_t mod_base = (size_t)m * p.module_px;
        const uint16_t* fr = raw + (size_t)f * p.frame_px + mod_base;
        const float* npm = p.nped + mod_base;
        const float* gm = p.inv_gain + mod_base;

        // ---- A. histogram of d per unit, code bytes kept -----------------
        if (median) {
            for (uint32_t i = tid; i < U * kFuHistWords / 4; i += nthr)
                reinterpret_cast<uint4*>(regb)[i] = make_uint4(0, 0, 0, 0);
        }
        if (tid < kFusedMaxUnits) {
            sh.s_cand[tid] = 0;
            sh.s_cm[tid] = 0.0f;
        }
        __syncthreads();  // also: the previous item's pass C is done with region A
                          // and with the seed-list counters
        if (tid == 0) sh.s_list[0] = 0;
        if (median) {
            const float2 eight = make_float2(8.0f, 8.0f);
            const float2 mw = make_float2(fc.magic_w, fc.magic_w);
            constexpr int UR = PD_FUSED_UNROLL;
            int r = active ? (int)ty : R;
            for (; r < R; r += UR * (int)TY) {
                uint2 x[UR];
                float4 np[UR];
#pragma unroll
                for (int j = 0; j < UR; j++) {
                    const int rr = r + j * (int)TY;
                    if (rr < R) {
                        const uint32_t off = (uint32_t)rr * (uint32_t)C + c4;
                        x[j] = *reinterpret_cast<const uint2*>(fr + off);
                        np[j] = *reinterpret_cast<const float4*>(npm + off);
                    }
                }
#pragma unroll
                for (int j = 0; j < UR; j++) {
                    const int rr = r + j * (int)TY;
                    if (rr >= R) break;
                    const float2 d01 = __fadd2_rn(raw_pair(x[j].x), make_float2(np[j].x, np[j].y));
                    const float2 d23 = __fadd2_rn(raw_pair(x[j].y), make_float2(np[j].z, np[j].w));
                    const float2 u01 = __ffma2_rd(d01, eight, mw);
                    const float2 u23 = __ffma2_rd(d23, eight, mw);
                    const int lo = (int)kMagicBits, hi = (int)(kMagicBits + kFuBins);
                    const uint32_t b0 = (uint32_t)min(max(__float_as_int(u01.x), lo), hi);
                    const uint32_t b1 = (uint32_t)min(max(__float_as_int(u01.y), lo), hi);
                    const uint32_t b2 = (uint32_t)min(max(__float_as_int(u23.x), lo), hi);
                    const uint32_t b3 = (uint32_t)min(max(__float_as_int(u23.y), lo), hi);
                    red_shared_add1(hb[0] + 4u * b0);
                    red_shared_add1(hb[1] + 4u * b1);
                    red_shared_add1(hb[2] + 4u * b2);
                    red_shared_add1(hb[3] + 4u * b3);
                    // low bytes (kMagicBits has a zero low byte)
                    codes32[(uint32_t)rr * TX + tx] =
                        __byte_perm(__byte_perm(b0, b1, 0x0040u), __byte_perm(b2, b3, 0x0040u),
                                    0x5410u);
                }
            }
        }
        __syncthreads();

        // ---- B. lower median per unit ------------------------------------
        if (median) {
            for (uint32_t g = tid; g < U * kFuGroups; g += nthr) {
                const uint32_t u = g / kFuGroups, gg = g % kFuGroups;
                const uint4* h4 = reinterpret_cast<const uint4*>(regb + u * kFuHistWords + gg * 32);
                uint32_t s = 0;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const uint4 v = h4[j];
                    s += v.x + v.y + v.z + v.w;
                }
                sh.gsum[u][gg] = s;
            }
            __syncthreads();
            if (warp < (int)U) {
                const uint32_t u = (uint32_t)warp;
                uint32_t loc[4], sum = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const uint32_t g = (uint32_t)lane * 4 + j;
                    loc[j] = g < kFuGroups ? sh.gsum[u][g] : 0u;
                    sum += loc[j];
                }
                uint32_t incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
                const bool enough = total > 0 && total >= p.cm_min_count;
                const uint32_t k = (total - 1) / 2;
                const uint32_t excl = incl - sum;
                const bool mine = enough && excl <= k && k < incl;
                const uint32_t who = __ballot_sync(0xffffffffu, mine);
                uint32_t group = 0, grank = 0;
                if (mine) {
                    uint32_t below = excl;
                    int gj = 0;
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if (below + loc[j] > k) {
                            gj = j;
                            break;
                        }
                        below += loc[j];
                    }
                    group = (uint32_t)lane * 4 + gj;
                    grank = k - below;
                }
                if (lane == 0) {
                    sh.s_n[u] = total;
                    sh.s_bin[u] = enough ? kFuBins : kFuBins + 1;  // +1: common mode 0
                }
                __syncwarp();
                if (enough) {
                    const int src = __ffs(who) - 1;
                    group = __shfl_sync(0xffffffffu, group, src);
                    grank = __shfl_sync(0xffffffffu, grank, src);
                    const uint32_t hv = regb[u * kFuHistWords + group * 32 + lane];
                    uint32_t hi = hv;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t v = __shfl_up_sync(0xffffffffu, hi, o);
                        if (lane >= o) hi += v;
                    }
                    const uint32_t he = hi - hv;
                    if (he <= grank && grank < hi) {
                        sh.s_bin[u] = group * 32 + lane;
                        sh.s_rank[u] = grank - he;
                    }
                }
            }
            __syncthreads();

            // units whose median bin is a closed bin take the candidate path
            uint32_t tw = 0, am = 0;
            bool any = false;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const uint32_t b = sh.s_bin[unit_of[i]];
                const bool cp = b >= 1 && b < kFuBins;
                tw |= (b & 0xFFu) << (8 * i);
                am |= cp ? (0x80u << (8 * i)) : 0u;
            }
            for (uint32_t u = 0; u < U; u++) {
                const uint32_t b = sh.s_bin[u];
                any = any || (b >= 1 && b < kFuBins);
            }
            bool pos_ok = true;
            if (any) {
                uint32_t mine = 0;
                for (int r = active ? (int)ty : R; r < R; r += (int)TY)
                    mine += __popc(zero_bytes(codes32[(uint32_t)r * TX + tx] ^ tw) & am);
                uint32_t at = block_excl_scan(mine, sh.swarp, &sh.s_pos);
                if (mine) {
                    for (int r = (int)ty; r < R && at < kFuPosCap; r += (int)TY) {
                        uint32_t z = zero_bytes(codes32[(uint32_t)r * TX + tx] ^ tw) & am;
                        while (z && at < kFuPosCap) {
                            const int i = (__ffs((int)z) - 1) >> 3;
                            z &= z - 1;
                            pos[at++] = (uint32_t)r * (uint32_t)C + c4 + (uint32_t)i;
                        }
                    }
                }
                __syncthreads();
                const uint32_t npos = sh.s_pos;
                pos_ok = npos <= kFuPosCap;
                if (pos_ok) {
                    // recompute d of every match and keep the true members
                    for (uint32_t t = tid; t < npos; t += nthr) {
                        const uint32_t px = pos[t];
                        const uint32_t u = (px % (uint32_t)C) / p.unit_cols;
                        const float d = __fadd_rn(raw_at(fr, px), npm[px]);
                        const uint32_t b = (uint32_t)fu_code(d, fc.magic_w) - kMagicBits;
                        if (b == sh.s_bin[u]) {
                            const uint32_t k = atomicAdd(&sh.s_cand[u], 1u);
                            if (k < cap_u) cand[u * cap_u + k] = d;
                        }
                    }
                }
                __syncthreads();
            }
            for (uint32_t u = 0; u < U; u++) {
                const uint32_t bin = sh.s_bin[u];
                if (bin > kFuBins) continue;  // fewer than the minimum count: 0
                const uint32_t mc = sh.s_cand[u];
                if (bin >= 1 && bin < kFuBins && pos_ok && mc <= cap_u) {
                    // exact select inside the bin: sub-bins of 1/8192 ADU
                    // (d - lo rounded to nearest is monotone in d), then
                    // counting among the values of the target sub-bin
                    const float* cu = cand + u * cap_u;
                    uint32_t* subcode = codes32;  // region A is free now
                    float* few = reinterpret_cast<float*>(pos);
                    const float lo_b = __fadd_rn(fc.w_lo, __fmul_rn((float)bin, 0.125f));
                    for (uint32_t i = tid; i < 1024 / 4; i += nthr)
                        reinterpret_cast<uint4*>(sub)[i] = make_uint4(0, 0, 0, 0);
                    if (tid == 0) sh.s_rrank = 0;
                    __syncthreads();
                    for (uint32_t t = tid; t < mc; t += nthr) {
                        const float x = __fmul_rn(__fsub_rn(cu[t], lo_b), 8192.0f);
                        const uint32_t sb = min((uint32_t)max(__float2int_rd(x), 0), 1023u);
                        subcode[t] = sb;
                        atomicAdd(&sub[sb], 1u);
                    }
                    __syncthreads();
                    const uint32_t brank = sh.s_rank[u];
                    find_rank<1024>(
                        sub, [brank](uint32_t) { return brank; }, sh.gsum[0], &sh.s_total,
                        &sh.s_sbin, &sh.s_srank);
                    const uint32_t sbin = sh.s_sbin, srank = sh.s_srank;
                    for (uint32_t t = tid; t < mc; t += nthr)
                        if (subcode[t] == sbin) few[atomicAdd(&sh.s_rrank, 1u)] = cu[t];
                    __syncthreads();
                    const uint32_t nf = sh.s_rrank;
                    for (uint32_t t = tid; t < nf; t += nthr) {
                        const uint32_t kt = order_key(few[t]);
                        uint32_t less = 0, leq = 0;
                        for (uint32_t j = 0; j < nf; j++) {
                            const uint32_t kj = order_key(few[j]);
                            less += kj < kt;
                            leq += kj <= kt;
                        }
                        if (less <= srank && srank < leq) sh.s_cm[u] = few[t];
                    }
                    __syncthreads();
                } else {
                    // whole-unit exact selection (bottom bin or overflow)
                    const uint32_t n = sh.s_n[u];
                    const uint32_t uc = p.unit_cols, col0 = u * uc;
                    const float cut = p.cm_cut;
                    auto key_at = [&](uint32_t i) -> uint32_t {
                        const uint32_t off = (i / uc) * (uint32_t)C + col0 + i % uc;
                        const float d = __fadd_rn(raw_at(fr, off), npm[off]);
                        return d < cut ? order_key(d) : kSent;
                    };
                    const uint32_t key = block_radix_select(key_at, p.unit_px, (n - 1) / 2, sub,
                                                            &sh.s_prefix, &sh.s_rrank);
                    if (tid == 0) sh.s_cm[u] = key_value(key);
                    __syncthreads();
                }
            }
        }
        if (out.cm && tid < p.units_per_module)
            out.cm[(size_t)f * p.units_per_frame + (size_t)m * p.units_per_module + tid] =
                median ? sh.s_cm[tid] : 0.0f;

        // ---- C. correction and stencil sweep -----------------------------
        // ring row of module row r: (r + 2) % kFuRing; rows -2 and -1 are
        // zero, and so are the 4 pad columns on each side of every row
        for (uint32_t i = tid; i < 2 * P; i += nthr) ring[i] = 0.0f;
        for (uint32_t i = tid; i < (kFuRing - 2) * 8; i += nthr) {
            const uint32_t row = 2 + i / 8, k = i % 8;
            ring[row * P + (k < 4 ? k : (uint32_t)C + k)] = 0.0f;
        }
        float ncm[4];
#pragma unroll
        for (int i = 0; i < 4; i++) ncm[i] = -sh.s_cm[unit_of[i]];
        __syncthreads();

        const float zt = p.zero_thr, st = p.seed_thr;
        const uint32_t BR = 2 * TY;
        uint32_t carry = 0;  // candidates of row r0 - 1 (thread ty == TY - 1)
        uint32_t band = 0;
        // loads of the next band are issued before the current band's seed
        // test, so they are in flight during it
        uint2 px[2];
        float4 pn[2], pg[2];
        auto load_band = [&](int rb0) {
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const int r = rb0 + (int)ty + j * (int)TY;
                if (active && r < R) {
                    const uint32_t off = (uint32_t)r * (uint32_t)C + c4;
                    px[j] = *reinterpret_cast<const uint2*>(fr + off);
                    pn[j] = *reinterpret_cast<const float4*>(npm + off);
                    pg[j] = *reinterpret_cast<const float4*>(gm + off);
                }
            }
        };
        load_band(0);
        for (int r0 = 0; r0 < R; r0 += (int)BR, band++) {
            const bool last = r0 + (int)BR >= R;
            const int t1 = last ? R : r0 + (int)BR - 1;  // rows tested: [r0 - 1, t1)
            uint32_t bits = carry;                       // bits 0-3: row r0 - 1
            uint32_t next_carry = 0;
#pragma unroll
            for (int j = 0; j < 2; j++) {
                if (!active) break;
                const int r = r0 + (int)ty + j * (int)TY;
                float* srow = ring + (uint32_t)((r + 2) % (int)kFuRing) * P + 4 + c4;
                if (r >= R) {
                    if (r < r0 + (int)BR) *reinterpret_cast<float4*>(srow) = make_float4(0, 0, 0, 0);
                    continue;
                }
                const float2 d01 = __fadd2_rn(raw_pair(px[j].x), make_float2(pn[j].x, pn[j].y));
                const float2 d23 = __fadd2_rn(raw_pair(px[j].y), make_float2(pn[j].z, pn[j].w));
                const float2 e01 = __fmul2_rn(__fadd2_rn(d01, make_float2(ncm[0], ncm[1])),
                                              make_float2(pg[j].x, pg[j].y));
                const float2 e23 = __fmul2_rn(__fadd2_rn(d23, make_float2(ncm[2], ncm[3])),
                                              make_float2(pg[j].z, pg[j].w));
                const float2 u01 = __fadd2_rd(__ffma2_rn(e01, iw, nl), mg);
                const float2 u23 = __fadd2_rd(__ffma2_rn(e23, iw, nl), mg);
                const int lo = (int)kMagicBits;
                atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u01.x), lo), max_bits) - kMagicBits], 1u);
                atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u01.y), lo), max_bits) - kMagicBits], 1u);
                atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u23.x), lo), max_bits) - kMagicBits], 1u);
                atomicAdd(&hpix[(uint32_t)min(max(__float_as_int(u23.y), lo), max_bits) - kMagicBits], 1u);
                const float e[4] = {e01.x, e01.y, e23.x, e23.y};
                float sv[4];
                uint32_t c = 0;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    sv[i] = e[i] > zt ? e[i] : 0.0f;
                    c |= (sv[i] > st ? 1u : 0u) << i;
                }
                *reinterpret_cast<float4*>(srow) = make_float4(sv[0], sv[1], sv[2], sv[3]);
                if (out.corrected) {
                    float* dst = out.corrected + (size_t)f * p.frame_px + mod_base +
                                 (uint32_t)r * (uint32_t)C + c4;
                    *reinterpret_cast<float4*>(dst) = make_float4(e[0], e[1], e[2], e[3]);
                }
                if (r < t1)
                    bits |= c << (4 + 4 * j);
                else
                    next_carry = c;  // the band's last row: tested with the next band
            }
            if (!last) load_band(r0 + (int)BR);
            if (last && r0 + (int)BR == R)  // row R reads as zero
                for (uint32_t i = tid; i < (uint32_t)C; i += nthr)
                    ring[(uint32_t)((R + 2) % (int)kFuRing) * P + 4 + i] = 0.0f;
            carry = next_carry;

            // compaction of the candidates into list band % 3
            const uint32_t li = band % 3;
            {
                const uint32_t cnt = __popc(bits);
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                uint32_t base = 0;
                if (lane == 31 && incl) base = atomicAdd(&sh.s_list[li], incl);
                base = __shfl_sync(0xffffffffu, base, 31);
                uint32_t at = base + incl - cnt;
                uint32_t* lst = lists + li * kFuListCap;
                while (bits) {
                    const int b = __ffs((int)bits) - 1;
                    bits &= bits - 1;
                    const int g = b >> 2;  // 0: row r0 - 1, 1: first row, 2: second row
                    const int r = g == 0 ? r0 - 1 : r0 + (int)ty + (g - 1) * (int)TY;
                    if (at < kFuListCap) lst[at] = ((uint32_t)r << 16) | (c4 + (uint32_t)(b & 3));
                    at++;
                }
            }
            if (tid == 0) sh.s_list[(band + 1) % 3] = 0;
            __syncthreads();

            // seeds: local maximum test, sums, count, centroid, emission
            const uint32_t n_list = sh.s_list[li];
            const bool scan = n_list > kFuListCap;  // overflow: test every pixel
            const int ta = max(r0 - 1, 0);
            const uint32_t n_work = scan ? (uint32_t)(t1 - ta) * (uint32_t)C : n_list;
            const uint32_t* lst = lists + li * kFuListCap;
            for (uint32_t b0 = 0; b0 < n_work; b0 += nthr) {
                const uint32_t j = b0 + tid;
                bool emit = false;
                pd_hit h;
                uint32_t n = 0, pix = 0;
                if (j < n_work) {
                    int r, c;
                    if (scan) {
                        r = ta + (int)(j / (uint32_t)C);
                        c = (int)(j % (uint32_t)C);
                    } else {
                        const uint32_t e = lst[j];
                        r = (int)(e >> 16);
                        c = (int)(e & 0xFFFFu);
                    }
                    const float* mid = ring + (uint32_t)((r + 2) % (int)kFuRing) * P + 4 + c;
                    const float* up = ring + (uint32_t)((r + 1) % (int)kFuRing) * P + 4 + c;
                    const float* dn = ring + (uint32_t)((r + 3) % (int)kFuRing) * P + 4 + c;
                    const float sp = mid[0];
                    if (sp > st) {
                        const float nb[9] = {up[-1],  up[0], up[1], mid[-1], sp,
                                             mid[1],  dn[-1], dn[0], dn[1]};
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
                                if (r == 0 || c == 0 || r == R - 1 || c == C - 1) flags |= PD_HIT_EDGE;
                                pix = (uint32_t)mod_base + (uint32_t)r * (uint32_t)C + (uint32_t)c;
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
        }
    }
    __syncthreads();
    for (uint32_t b = tid; b < p.hist_bins; b += nthr) {
        if (hpix[b]) atomicAdd(&p.hist_pix[b], (unsigned long long)hpix[b]);
        if (hhit[b]) atomicAdd(&p.hist_hit[b], (unsigned long long)hhit[b]);
    }
}

FusedConfig make_fused_config(const ChainParams& p) {
    FusedConfig fc{};
    fc.ok = false;
    if (p.cols % 4 != 0 || p.cols / 4 > 512 || p.cols >= 65536 || p.rows >= 65536) return fc;
    const bool median = cm_kind(p) == PD_CM_MEDIAN;
    if (median) {
        if (p.unit_rows != p.rows || p.units_per_row > kFusedMaxUnits) return fc;
        const double cut = p.cm_cut;
        const double lo8 = (cut - 448.0) * 8.0;
        if (!(cut > -1e6 && cut < 1e6) || lo8 != (double)(long long)lo8) return fc;
        fc.magic_w = (float)(12582912.0 - lo8);
        fc.w_lo = (float)(cut - 448.0);
        if ((double)fc.magic_w != 12582912.0 - lo8) return fc;
    } else if (p.units_per_module > 512) {
        return fc;
    }
    fc.tx = p.cols / 4;
    // each band is 2 * ty rows; the ring needs 2 * (2 * ty) + 2 <= kFuRing
    fc.ty = std::min<uint32_t>(std::max<uint32_t>(1, 512 / fc.tx), kFusedMaxTy);
    if (fc.tx * fc.ty < std::max<uint32_t>(p.units_per_module, kFusedMaxUnits)) return fc;
    fc.pitch = p.cols + 8;
    const uint32_t a_words = std::max<uint32_t>((p.module_px + 3) / 4,
                                                kFuRing * fc.pitch + 3 * kFuListCap);
    fc.region_a_words = (a_words + 3) / 4 * 4;
    const uint32_t b_words = std::max<uint32_t>(kFusedMaxUnits * kFuHistWords,
                                                kFuPosCap + kFuCandCap + 1024);
    fc.region_b_words = (b_words + 3) / 4 * 4;
    fc.smem_bytes = (fc.region_a_words + fc.region_b_words + 2 * p.hist_bins + 4) * 4;
    fc.ok = fc.smem_bytes <= 200 * 1024;
    return fc;
}

static int g_attr_dev_fused = -1;

template <int MAXT>
static cudaError_t launch_fused_t(const ChainParams& p, const FusedConfig& fc,
                                  const uint16_t* raw, uint32_t n_frames, uint32_t frame_base,
                                  const CallOut& out, cudaStream_t stream, unsigned threads,
                                  unsigned long long items) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, chain_module_kernel<MAXT>, (int)threads, fc.smem_bytes);
    if (e != cudaSuccess) return e;
    const unsigned long long grid =
        std::min<unsigned long long>(items, (unsigned long long)std::max(per_sm, 1) *
                                                (unsigned long long)device_sm_count());
    chain_module_kernel<MAXT><<<(unsigned)grid, threads, fc.smem_bytes, stream>>>(
        p, fc, raw, n_frames, frame_base, out);
    return cudaGetLastError();
}

cudaError_t launch_fused(const ChainParams& p, const FusedConfig& fc, const uint16_t* raw,
                         uint32_t n_frames, uint32_t frame_base, const CallOut& out,
                         cudaStream_t stream) {
    const unsigned long long items = (unsigned long long)n_frames * p.n_modules;
    if (items == 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_attr_dev_fused != dev) {
        cudaError_t e = cudaFuncSetAttribute(chain_module_kernel<320>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(chain_module_kernel<512>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        g_attr_dev_fused = dev;
    }
    const unsigned threads = (fc.tx * fc.ty + 31) / 32 * 32;
    return threads <= 320
               ? launch_fused_t<320>(p, fc, raw, n_frames, frame_base, out, stream, threads, items)
               : launch_fused_t<512>(p, fc, raw, n_frames, frame_base, out, stream, threads, items);
}

}  // namespace pd
