// pd_dev.cuh — device helpers shared by the throughput kernels: exact
// float <-> order-preserving key maps, floor-by-magic-number bin codes,
// packed raw conversion, and block-wide scan / select / rank location.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pd {
namespace {

constexpr uint32_t kSent = 0xFFFFFFFFu;
constexpr uint32_t kMagicBits = 0x4B400000u;  // bit pattern of 1.5 * 2^23
constexpr float kMagic = 12582912.0f;         // 1.5 * 2^23

__device__ __forceinline__ uint32_t order_key(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_value(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}


// Band, module and frame of tiles t, t + step, t + 2 step, ... of a band
// stencil (tile t is band t % nb of module (t / nb) % nm of frame
// t / (nb nm)), split once and then advanced with carries instead of 64-bit
// divisions per tile.
struct TileWalk {
    uint32_t band, m, f;     // of the current tile
    uint32_t sb, sm, sf;     // the step split the same way
    uint32_t nb, nm;
    __device__ __forceinline__ TileWalk(unsigned long long t, unsigned long long step,
                                        uint32_t n_bands, uint32_t n_modules)
        : nb(n_bands), nm(n_modules) {
        band = (uint32_t)(t % nb);
        t /= nb;
        m = (uint32_t)(t % nm);
        f = (uint32_t)(t / nm);
        sb = (uint32_t)(step % nb);
        step /= nb;
        sm = (uint32_t)(step % nm);
        sf = (uint32_t)(step / nm);
    }
    __device__ __forceinline__ void next() {
        band += sb;
        const uint32_t cb = band >= nb;
        if (cb) band -= nb;
        m += sm + cb;  // below 2 nm
        const uint32_t cm = m >= nm;
        if (cm) m -= nm;
        f += sf + cm;
    }
};

// Bulk prefetch into L2 of the whole 16-byte units inside [a, b) (global
// addresses; nothing outside the range is touched, nothing to wait for).
__device__ __forceinline__ void prefetch_l2_range(const void* a, const void* b) {
    const uint64_t s = ((uint64_t)a + 15ull) & ~15ull, e = (uint64_t)b & ~15ull;
    if (e > s)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s))
                     : "memory");
}

// The raw rows of a band stencil's tile asked of L2: band w.band (rb rows)
// of module w.m of frame w.f, with the halo row above and `below` halo rows
// below where the module has them; mod_rows x cols words per module,
// frame_px per frame.
__device__ __forceinline__ void prefetch_tile_rows(const uint16_t* raw, const TileWalk& w,
                                                   uint32_t rb, uint32_t mod_rows, uint32_t cols,
                                                   size_t frame_px, int below = 1) {
    const int r0 = (int)(w.band * rb);
    const int ra = max(r0 - 1, 0), re = min(r0 + (int)rb + below, (int)mod_rows);
    const uint16_t* mod = raw + (size_t)w.f * frame_px + (size_t)w.m * mod_rows * cols;
    prefetch_l2_range(mod + (size_t)ra * cols, mod + (size_t)re * cols);
}

// Histogram bin of the summaries: floor(fma(v, inv_w, -lo_s)) clipped to
// [0, bins-1], as the code of an element of a 32-bit histogram array.
__device__ __forceinline__ uint32_t summary_bin(float v, float inv_w, float neg_lo_s,
                                                int max_bits) {
    const float t = __fmaf_rn(v, inv_w, neg_lo_s);
    int b = __float_as_int(__fadd_rd(t, kMagic));
    b = max(b, (int)kMagicBits);
    b = min(b, max_bits);
    return (uint32_t)(b - (int)kMagicBits);
}

// Centroid offset m / e rounded to nearest (section "Photon Subpixel
// Resolution").  A zero moment over a positive energy is that zero, sign
// included, exactly as the division gives it; testing for it first keeps
// single-pixel hits (both moments zero) off the division's slow path.
__device__ __forceinline__ float moment_over_energy(float m, float e) {
    return m == 0.0f && e > 0.0f ? m : __fdiv_rn(m, e);
}

// Two raw values of a packed pair as exact floats: 2^23 + raw has the raw
// value as its low mantissa bits, and subtracting 2^23 is exact.
__device__ __forceinline__ float2 raw_pair(uint32_t x) {
    const float2 biased = make_float2(__uint_as_float(__byte_perm(x, 0x4B00u, 0x5410u)),
                                      __uint_as_float(__byte_perm(x, 0x4B00u, 0x5432u)));
    return __fadd2_rn(biased, make_float2(-8388608.0f, -8388608.0f));
}

// Common-mode bin code of d: floor(8 * (d - lo)) clipped below at 0 and
// above at 0xFFFF; codes >= kCmBins mean d >= cut (anchored window).
__device__ __forceinline__ uint32_t cm_code(float d, float magic_w) {
    int b = __float_as_int(__fmaf_rd(d, 8.0f, magic_w));
    b = max(b, (int)kMagicBits);
    b = min(b, (int)(kMagicBits + 0xFFFFu));
    return (uint32_t)(b - (int)kMagicBits);
}

// Asynchronous 4-byte global -> shared copy (no register staging), and the
// wait for all of this thread's copies.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// Block-wide exact radix select: the element of rank `rank` (0-based,
// ascending) among the keys key_at(i), i < count, that are not kSent.
// hist256: 256 words of shared memory.  All threads must call it.
template <class KeyFn>
__device__ uint32_t block_radix_select(KeyFn key_at, uint32_t count, uint32_t rank,
                                       uint32_t* hist256, uint32_t* s_prefix,
                                       uint32_t* s_rank) {
    const uint32_t nthr = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        *s_prefix = 0;
        *s_rank = rank;
    }
    for (int pass = 0; pass < 4; pass++) {
        const int shift = 24 - 8 * pass;
        for (uint32_t b = tid; b < 256; b += nthr) hist256[b] = 0;
        __syncthreads();
        const uint32_t prefix = *s_prefix;
        for (uint32_t i = tid; i < count; i += nthr) {
            const uint32_t k = key_at(i);
            if (k == kSent) continue;
            if (pass > 0 && (k >> (shift + 8)) != prefix) continue;
            atomicAdd(&hist256[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t loc[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                loc[j] = hist256[lane * 8 + j];
                sum += loc[j];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t excl = incl - sum;
            const uint32_t r = *s_rank;
            if (excl <= r && r < incl) {
                uint32_t below = excl;
                int digit = lane * 8;
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    if (below + loc[j] > r) {
                        digit = lane * 8 + j;
                        break;
                    }
                    below += loc[j];
                }
                *s_prefix = (prefix << 8) | (uint32_t)digit;
                *s_rank = r - below;
            }
        }
        __syncthreads();
    }
    return *s_prefix;
}

// Block-wide exclusive prefix sum of one value per thread; *s_total gets the
// sum.  s_warp: 32 words of shared memory.  All threads must call it.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp,
                                                    uint32_t* s_total) {
    const uint32_t tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31 || tid == blockDim.x - 1) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nwarps ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += x;
        }
        if (lane < nwarps) s_warp[lane] = wi - w;
        if (lane == 31) *s_total = wi;
    }
    __syncthreads();
    return s_warp[warp] + incl - v;
}

// ---------------------------------------------------------------------------
// Block-wide location of a rank in a histogram of NB bins (NB = 1024 * G):
// sums of 32-bin groups, then one warp scans the group sums and the group.
// target_of(total) gives the rank to find (or total or more for none).
// Results in *s_total, *s_bin, *s_rank (rank within the bin); *s_bin = NB
// when no bin holds the target.  All threads must call it.
template <int NB, class TargetFn>
__device__ void find_rank(const uint32_t* hist, TargetFn target_of, uint32_t* gsum,
                          uint32_t* s_total, uint32_t* s_bin, uint32_t* s_rank) {
    constexpr int NG = NB / 32;  // groups
    constexpr int G = NG / 32;   // groups per lane
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    for (uint32_t g = tid; g < (uint32_t)NG; g += nthr) {
        const uint4* h4 = reinterpret_cast<const uint4*>(hist + g * 32);
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint4 v = h4[j];
            sum += v.x + v.y + v.z + v.w;
        }
        gsum[g] = sum;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t loc[G], sum = 0;
#pragma unroll
        for (int j = 0; j < G; j++) {
            loc[j] = gsum[lane * G + j];
            sum += loc[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t k = target_of(total);
        const bool ok = k < total;
        const uint32_t excl = incl - sum;
        const bool mine = ok && excl <= k && k < incl;
        const uint32_t who = __ballot_sync(0xffffffffu, mine);
        uint32_t group = 0, grank = 0;
        if (mine) {
            uint32_t below = excl;
            int gj = 0;
#pragma unroll
            for (int j = 0; j < G; j++) {
                if (below + loc[j] > k) {
                    gj = j;
                    break;
                }
                below += loc[j];
            }
            group = lane * G + gj;
            grank = k - below;
        }
        if (lane == 0) {
            *s_total = total;
            *s_bin = NB;
        }
        __syncwarp();
        if (ok) {
            const int src = __ffs(who) - 1;
            group = __shfl_sync(0xffffffffu, group, src);
            grank = __shfl_sync(0xffffffffu, grank, src);
            const uint32_t hv = hist[group * 32 + lane];
            uint32_t hi = hv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, hi, o);
                if (lane >= o) hi += v;
            }
            const uint32_t he = hi - hv;
            if (he <= grank && grank < hi) {
                *s_bin = group * 32 + lane;
                *s_rank = grank - he;
            }
        }
    }
    __syncthreads();
}

}  // namespace
}  // namespace pd
