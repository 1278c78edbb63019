// pd_cm_mean.cu — the paper's common-mode estimator and its stacked stages.
//
// Section "Common Mode" and Fig. c: the pixels of a group whose value v is
// below the noise cut are counted (N0) and summed (S), and the group's common
// mode is S / max(N0, sqrt(G)) with G the group's pixel count; the sqrt(G)
// term keeps a group with few background pixels from being corrected by a
// noisy estimate.  The same section obtains row, column and block variants by
// summing over other groups, and section "Performance" stacks three
// common-mode stages.  Here:
//
//   PD_CM_MEAN           one stage over each unit (v = d = raw - pedestal)
//   PD_CM_MEAN_STACKED   unit, then each module row on d - cm_u, then each
//                        module column on (d - cm_u) - cm_r
//
// S is defined independently of the summation order, so that any grid gives
// the same bits: with M the largest |v| of the selected values and
// E = max(floor(log2 M), -60), each v is rounded to the grid 2^(E-38)
// (round to nearest even) as a 64-bit integer, the integers are added
// exactly, and the total is rounded once to binary32.  Values down to
// M * 2^-15 lie on the grid, so for detector data S is the exactly rounded
// sum.  Each group takes two passes over its pixels: count and largest
// magnitude, then the integer sum.
//
// Kernels (the second and third only for the stacked mode):
//   mean_units_block_kernel  one CTA per (frame, unit) for units of 8+ rows
//   mean_units_warp_kernel   one warp per (frame, unit) for shorter units
//   mean_rows_kernel         one warp per (frame, module, row)
//   mean_cols_kernel         one warp per (frame, module, 32 columns), one
//                            lane per column walking down the rows
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kMeanThreads = 256;
constexpr int kMeanWarps = kMeanThreads / 32;

__device__ __forceinline__ bool selects(float v, float cut) {
    return v < cut && v > -INFINITY;
}

__device__ __forceinline__ uint32_t abs_bits(float v) { return __float_as_uint(v) & 0x7fffffffu; }

// 2^k as a float for -126 < k < 128
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(127 + k) << 23); }

// grid exponent: the values are scaled by 2^k before rounding to integers
__device__ __forceinline__ int grid_k(uint32_t max_bits) {
    int e = (int)(max_bits >> 23) - 127;  // floor(log2 M); subnormal M gives -127
    if (e < -60) e = -60;
    return 38 - e;
}

struct Acc {
    uint32_t n0 = 0, max_bits = 0;
    long long total = 0;

    __device__ __forceinline__ void first(float v, float cut) {
        if (selects(v, cut)) {
            n0++;
            max_bits = max(max_bits, abs_bits(v));
        }
    }
    __device__ __forceinline__ void second(float v, float cut, float scale) {
        if (selects(v, cut)) total += __float2ll_rn(__fmul_rn(v, scale));
    }
};

__device__ __forceinline__ float mean_of(long long total, uint32_t n0, uint32_t max_bits,
                                         float guard) {
    float sum = 0.0f;
    if (n0 > 0 && max_bits != 0) sum = __fmul_rn(__ll2float_rn(total), pow2f(-grid_k(max_bits)));
    return __fdiv_rn(sum, fmaxf((float)n0, guard));
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float dark(const uint16_t* raw, const float* nped, size_t off) {
    return __fadd_rn(__uint2float_rn(raw[off]), nped[off]);
}

// A pixel's common-mode input: d, or in the paper's order d * inv_gain (NaN
// for masked pixels, which no selection takes).
__device__ __forceinline__ float cmv(bool ag, const uint16_t* raw, const float* nped,
                                     const float* ig, size_t off) {
    const float d = dark(raw, nped, off);
    return ag ? cm_input(true, d, ig[off]) : d;
}

// Offsets of frame f, unit u in the pixel arrays and its rectangle origin.
struct UnitAt {
    size_t raw_off, map_off;
};

__device__ __forceinline__ UnitAt unit_at(const ChainParams& p, uint32_t f, uint32_t u) {
    const uint32_t m = u / p.units_per_module, uu = u % p.units_per_module;
    const uint32_t r0 = (uu / p.units_per_row) * p.unit_rows;
    const uint32_t c0 = (uu % p.units_per_row) * p.unit_cols;
    const size_t map = (size_t)m * p.module_px + (size_t)r0 * p.cols + c0;
    return UnitAt{(size_t)f * p.frame_px + map, map};
}

// ---------------------------------------------------------------------------
// stage 1, units of at least 8 rows: warps over rows, lanes over columns
__global__ void __launch_bounds__(kMeanThreads)
    mean_units_block_kernel(ChainParams p, const uint16_t* __restrict__ raw,
                            float* __restrict__ cm) {
    __shared__ uint32_t s_n0, s_max;
    __shared__ unsigned long long s_total;
    const uint32_t f = blockIdx.x / p.units_per_frame, u = blockIdx.x % p.units_per_frame;
    const UnitAt at = unit_at(p, f, u);
    const uint16_t* rw = raw + at.raw_off;
    const float* np_ = p.nped + at.map_off;
    const float* ig_ = p.inv_gain + at.map_off;
    const bool ag = cm_after_gain(p);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_n0 = 0;
        s_max = 0;
        s_total = 0;
    }
    __syncthreads();
    Acc a;
    for (uint32_t r = warp; r < p.unit_rows; r += kMeanWarps)
        for (uint32_t c = lane; c < p.unit_cols; c += 32) {
            const size_t off = (size_t)r * p.cols + c;
            a.first(cmv(ag, rw, np_, ig_, off), p.cm_cut);
        }
    const uint32_t wn = __reduce_add_sync(0xffffffffu, a.n0);
    const uint32_t wm = __reduce_max_sync(0xffffffffu, a.max_bits);
    if (lane == 0) {
        atomicAdd(&s_n0, wn);
        atomicMax(&s_max, wm);
    }
    __syncthreads();
    const uint32_t n0 = s_n0, mb = s_max;
    if (n0 > 0 && mb != 0) {
        const float scale = pow2f(grid_k(mb));
        for (uint32_t r = warp; r < p.unit_rows; r += kMeanWarps)
            for (uint32_t c = lane; c < p.unit_cols; c += 32) {
                const size_t off = (size_t)r * p.cols + c;
                a.second(cmv(ag, rw, np_, ig_, off), p.cm_cut, scale);
            }
        const long long wt = warp_sum64(a.total);
        if (lane == 0) atomicAdd(&s_total, (unsigned long long)wt);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        cm[(size_t)f * cm_per_frame(p) + u] =
            mean_of((long long)s_total, n0, mb, __fsqrt_rn((float)p.unit_px));
}

// stage 1, units of fewer than 8 rows: one warp per unit
__global__ void __launch_bounds__(kMeanThreads)
    mean_units_warp_kernel(ChainParams p, const uint16_t* __restrict__ raw,
                           float* __restrict__ cm, uint32_t n_units) {
    const uint32_t item = blockIdx.x * kMeanWarps + (threadIdx.x >> 5);
    if (item >= n_units) return;  // whole warps leave together
    const int lane = threadIdx.x & 31;
    const uint32_t f = item / p.units_per_frame;
    const uint32_t u = item % p.units_per_frame;
    const UnitAt at = unit_at(p, f, u);
    const uint16_t* rw = raw + at.raw_off;
    const float* np_ = p.nped + at.map_off;
    const float* ig_ = p.inv_gain + at.map_off;
    const bool ag = cm_after_gain(p);
    Acc a;
    for (uint32_t r = 0; r < p.unit_rows; r++)
        for (uint32_t c = lane; c < p.unit_cols; c += 32)
            a.first(cmv(ag, rw, np_, ig_, (size_t)r * p.cols + c), p.cm_cut);
    const uint32_t n0 = __reduce_add_sync(0xffffffffu, a.n0);
    const uint32_t mb = __reduce_max_sync(0xffffffffu, a.max_bits);
    long long total = 0;
    if (n0 > 0 && mb != 0) {
        const float scale = pow2f(grid_k(mb));
        for (uint32_t r = 0; r < p.unit_rows; r++)
            for (uint32_t c = lane; c < p.unit_cols; c += 32)
                a.second(cmv(ag, rw, np_, ig_, (size_t)r * p.cols + c), p.cm_cut, scale);
        total = warp_sum64(a.total);
    }
    if (lane == 0)
        cm[(size_t)f * cm_per_frame(p) + u] =
            mean_of(total, n0, mb, __fsqrt_rn((float)p.unit_px));
}

// ---------------------------------------------------------------------------
// stage 2: one warp per (frame, module, row), on d - cm_u
__global__ void __launch_bounds__(kMeanThreads)
    mean_rows_kernel(ChainParams p, const uint16_t* __restrict__ raw, float* __restrict__ cm,
                     uint32_t n_rows) {
    const uint32_t item = blockIdx.x * kMeanWarps + (threadIdx.x >> 5);
    if (item >= n_rows) return;
    const int lane = threadIdx.x & 31;
    const uint32_t r = item % p.rows;
    const uint32_t fm = item / p.rows;
    const uint32_t m = fm % p.n_modules, f = fm / p.n_modules;
    const size_t map = (size_t)m * p.module_px + (size_t)r * p.cols;
    const uint16_t* rw = raw + (size_t)f * p.frame_px + map;
    const float* np_ = p.nped + map;
    const float* ig_ = p.inv_gain + map;
    const bool ag = cm_after_gain(p);
    const float* cmf = cm + (size_t)f * cm_per_frame(p);
    const float* cmu = cmf + (size_t)m * p.units_per_module + (r / p.unit_rows) * p.units_per_row;
    Acc a;
    for (uint32_t j = 0; j < p.units_per_row; j++) {
        const float cu = cmu[j];
        for (uint32_t c = j * p.unit_cols + lane; c < (j + 1) * p.unit_cols; c += 32)
            a.first(__fsub_rn(cmv(ag, rw, np_, ig_, c), cu), p.cm_cut);
    }
    const uint32_t n0 = __reduce_add_sync(0xffffffffu, a.n0);
    const uint32_t mb = __reduce_max_sync(0xffffffffu, a.max_bits);
    long long total = 0;
    if (n0 > 0 && mb != 0) {
        const float scale = pow2f(grid_k(mb));
        for (uint32_t j = 0; j < p.units_per_row; j++) {
            const float cu = cmu[j];
            for (uint32_t c = j * p.unit_cols + lane; c < (j + 1) * p.unit_cols; c += 32)
                a.second(__fsub_rn(cmv(ag, rw, np_, ig_, c), cu), p.cm_cut, scale);
        }
        total = warp_sum64(a.total);
    }
    if (lane == 0)
        cm[(size_t)f * cm_per_frame(p) + p.units_per_frame + (size_t)m * p.rows + r] =
            mean_of(total, n0, mb, __fsqrt_rn((float)p.cols));
}

// stage 3: one warp per (frame, module, block of 32 columns), one lane per
// column, on (d - cm_u) - cm_r
__global__ void __launch_bounds__(kMeanThreads)
    mean_cols_kernel(ChainParams p, const uint16_t* __restrict__ raw, float* __restrict__ cm,
                     uint32_t col_blocks, uint32_t n_items) {
    const uint32_t item = blockIdx.x * kMeanWarps + (threadIdx.x >> 5);
    if (item >= n_items) return;
    const int lane = threadIdx.x & 31;
    const uint32_t cb = item % col_blocks;
    const uint32_t fm = item / col_blocks;
    const uint32_t m = fm % p.n_modules, f = fm / p.n_modules;
    const uint32_t c = cb * 32 + lane;
    if (c >= p.cols) return;  // lanes stay independent from here on
    const size_t map = (size_t)m * p.module_px + c;
    const uint16_t* rw = raw + (size_t)f * p.frame_px + map;
    const float* np_ = p.nped + map;
    const float* ig_ = p.inv_gain + map;
    const bool ag = cm_after_gain(p);
    const float* cmf = cm + (size_t)f * cm_per_frame(p);
    const float* cmu = cmf + (size_t)m * p.units_per_module + c / p.unit_cols;
    const float* cmr = cmf + p.units_per_frame + (size_t)m * p.rows;
    const uint32_t unit_blocks = p.rows / p.unit_rows;
    Acc a;
    for (uint32_t b = 0; b < unit_blocks; b++) {
        const float cu = cmu[(size_t)b * p.units_per_row];
        for (uint32_t r = b * p.unit_rows; r < (b + 1) * p.unit_rows; r++)
            a.first(__fsub_rn(__fsub_rn(cmv(ag, rw, np_, ig_, (size_t)r * p.cols), cu), cmr[r]),
                    p.cm_cut);
    }
    if (a.n0 > 0 && a.max_bits != 0) {
        const float scale = pow2f(grid_k(a.max_bits));
        for (uint32_t b = 0; b < unit_blocks; b++) {
            const float cu = cmu[(size_t)b * p.units_per_row];
            for (uint32_t r = b * p.unit_rows; r < (b + 1) * p.unit_rows; r++)
                a.second(__fsub_rn(__fsub_rn(cmv(ag, rw, np_, ig_, (size_t)r * p.cols), cu), cmr[r]),
                         p.cm_cut, scale);
        }
    }
    cm[(size_t)f * cm_per_frame(p) + p.units_per_frame + (size_t)p.n_modules * p.rows +
       (size_t)m * p.cols + c] = mean_of(a.total, a.n0, a.max_bits, __fsqrt_rn((float)p.rows));
}

unsigned warps_grid(unsigned long long items) {
    return (unsigned)((items + kMeanWarps - 1) / kMeanWarps);
}

}  // namespace

cudaError_t launch_cm_mean(const ChainParams& p, const uint16_t* raw, uint32_t n_frames,
                           float* cm, cudaStream_t stream) {
    if (n_frames == 0) return cudaSuccess;
    // frames in groups whose work items (units, module rows, column blocks)
    // stay below 2^31, so the kernels index them in 32 bits
    const uint64_t per_frame = std::max<uint64_t>(
        {(uint64_t)p.units_per_frame, (uint64_t)p.n_modules * p.rows,
         (uint64_t)p.n_modules * ((p.cols + 31) / 32), 1});
    const uint32_t group = (uint32_t)std::max<uint64_t>(1, ((1ull << 31) - 1) / per_frame);
    const uint32_t col_blocks = (p.cols + 31) / 32;
    for (uint32_t f0 = 0; f0 < n_frames; f0 += group) {
        const uint32_t nf = std::min(group, n_frames - f0);
        const uint16_t* fr = raw + (size_t)f0 * p.frame_px;
        float* cmf = cm + (size_t)f0 * cm_per_frame(p);
        const uint32_t units = nf * p.units_per_frame;
        if (p.unit_rows >= kMeanWarps)
            mean_units_block_kernel<<<units, kMeanThreads, 0, stream>>>(p, fr, cmf);
        else
            mean_units_warp_kernel<<<warps_grid(units), kMeanThreads, 0, stream>>>(p, fr, cmf,
                                                                                  units);
        if (cm_kind(p) != PD_CM_MEAN_STACKED) continue;
        const uint32_t rows = nf * p.n_modules * p.rows;
        mean_rows_kernel<<<warps_grid(rows), kMeanThreads, 0, stream>>>(p, fr, cmf, rows);
        const uint32_t cols = nf * p.n_modules * col_blocks;
        mean_cols_kernel<<<warps_grid(cols), kMeanThreads, 0, stream>>>(p, fr, cmf, col_blocks,
                                                                        cols);
    }
    return cudaGetLastError();
}

}  // namespace pd
