// pd_net.cu — the learned photon count / subpixel network: patch gather,
// forward, loss, backward and Adam, as hand-written kernels.
//
// The paper found off-the-shelf deep models lost photon information and
// offered its fixed filters as the seed of future learned models (abstract,
// sections "Methods" and "Conclusions").  This network refines the classical
// count and centre of mass of each hit from the 5x5 neighbourhood of its
// seed: conv3x3x32 -> conv3x3x32 -> FC64 -> {5 count logits, (dx, dy)}.
//
// Training runs every layer with a contraction as a GEMM on the tensor
// cores (mma.sync m16n8k16, bfloat16 operands rounded to nearest even,
// float32 accumulation); inference (pd_net_forward) runs on tcgen05 with
// TMEM accumulators (pd_net_tc.cu), with the same operand rounding.  Convolutions are implicit GEMMs: operand loaders read the
// 3x3 neighbourhood (zero padded) directly, so no im2col buffer exists.
// Biases, ReLU, the loss and the optimiser are float32.  Layouts follow the
// oracle (oracle/net.py): activations [hit][position 0..24][channel].
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <string>
#include <vector>

#include "pd.h"
#include "pd_internal.cuh"
#include "pd_net_tc.cuh"

namespace {

constexpr int NPOS = 25, C1 = 32, C2 = 32, NH = 64, NOUT = 7;
constexpr int NW1 = C1 * 9, NB1 = C1, NW2 = C2 * 9 * C1, NB2 = C2, NW3 = NH * NPOS * C2,
              NB3 = NH, NW4 = NOUT * NH, NB4 = NOUT;
constexpr int OW1 = 0, OB1 = OW1 + NW1, OW2 = OB1 + NB1, OB2 = OW2 + NW2, OW3 = OB2 + NB2,
              OB3 = OW3 + NW3, OW4 = OB3 + NB3, OB4 = OW4 + NW4, NPARAM = OB4 + NB4;

// ---------------------------------------------------------------------------
// Tensor-core GEMM: C[M][N] = sum_k A(i, k) * B(k, j), operands from loader
// functors, results to an epilogue functor ep(i, j, value).  Block tile
// 64 x 64 x 32, four warps of 32 x 32; grid.z splits K (the epilogue then
// accumulates atomically).
constexpr int BM = 64, BN = 64, BK = 32, GT = 128, PADK = BK + 8;

__device__ __forceinline__ uint16_t bf16_bits(float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&b);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <class LA, class LB, class EP>
__global__ void __launch_bounds__(GT)
    gemm_kernel(int M, int N, int K, int k_split, LA la, LB lb, EP ep) {
    __shared__ __align__(16) uint16_t As[BM][PADK];
    __shared__ __align__(16) uint16_t Bs[BN][PADK];  // transposed: [n][k]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * k_split, kend = min(K, kbeg + k_split);
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][b][c] = 0.0f;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int e = tid; e < BM * BK; e += GT) {
            const int r = e / BK, c = e % BK;
            const int gi = m0 + r, gk = k0 + c;
            As[r][c] = bf16_bits((gi < M && gk < kend) ? la(gi, gk) : 0.0f);
        }
        for (int e = tid; e < BN * BK; e += GT) {
            const int n = e / BK, c = e % BK;
            const int gj = n0 + n, gk = k0 + c;
            Bs[n][c] = bf16_bits((gj < N && gk < kend) ? lb(gk, gj) : 0.0f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; mi++) {
                const int row = wm + mi * 16 + g;
                af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[row][kk + 2 * tq]);
                af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[row + 8][kk + 2 * tq]);
                af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[row][kk + 8 + 2 * tq]);
                af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[row + 8][kk + 8 + 2 * tq]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ni++) {
                const int n = wn + ni * 8 + g;
                bfr[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * tq]);
                bfr[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 8 + 2 * tq]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; mi++)
#pragma unroll
                for (int ni = 0; ni < 4; ni++) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++) {
            const int r = m0 + wm + mi * 16 + g, c = n0 + wn + ni * 8 + 2 * tq;
            if (r < M && c < N) ep(r, c, acc[mi][ni][0]);
            if (r < M && c + 1 < N) ep(r, c + 1, acc[mi][ni][1]);
            if (r + 8 < M && c < N) ep(r + 8, c, acc[mi][ni][2]);
            if (r + 8 < M && c + 1 < N) ep(r + 8, c + 1, acc[mi][ni][3]);
        }
}

template <class LA, class LB, class EP>
cudaError_t gemm(int M, int N, int K, LA la, LB lb, EP ep, cudaStream_t s, int splits = 1) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    splits = std::max(1, std::min(splits, (K + BK - 1) / BK));
    int k_split = (K + splits - 1) / splits;
    k_split = (k_split + BK - 1) / BK * BK;
    splits = (K + k_split - 1) / k_split;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    gemm_kernel<<<grid, GT, 0, s>>>(M, N, K, k_split, la, lb, ep);
    return cudaGetLastError();
}

// ---- operand loaders --------------------------------------------------------
// 3x3 neighbour of position p (0..24 on the 5x5 grid) at offset k, or -1.
__device__ __forceinline__ int nbr(int p, int k) {
    const int y = p / 5 + k / 3 - 1, x = p % 5 + k % 3 - 1;
    return (y >= 0 && y < 5 && x >= 0 && x < 5) ? y * 5 + x : -1;
}

struct RowMajor {  // element (i, k) of a row-major matrix with leading dim ld
    const float* a;
    int ld;
    __device__ float operator()(int i, int k) const { return a[(size_t)i * ld + k]; }
};
struct ColMajor {  // element (i, k) = a[k][i]: the transpose of a row-major matrix
    const float* a;
    int ld;
    __device__ float operator()(int i, int k) const { return a[(size_t)k * ld + i]; }
};
struct Im2col {  // element ((hit, p), k*C + c) of the im2col of act [hit][25][C]
    const float* act;
    int C;
    __device__ float operator()(int row, int col) const {
        const int hit = row / NPOS, p = row % NPOS, k = col / C, c = col % C;
        const int q = nbr(p, k);
        return q < 0 ? 0.0f : act[((size_t)hit * NPOS + q) * C + c];
    }
};
// ---- epilogues -----------------------------------------------------------
struct BiasAct {  // out[i][j] = act(acc + bias[j])
    float* out;
    int ld;
    const float* bias;
    bool relu;
    __device__ void operator()(int i, int j, float v) const {
        v = v + bias[j];
        out[(size_t)i * ld + j] = relu ? fmaxf(v, 0.0f) : v;
    }
};
struct ReluGrad {  // out[i][j] = acc * (act[i][j] > 0)
    float* out;
    const float* act;
    int ld;
    __device__ void operator()(int i, int j, float v) const {
        const size_t o = (size_t)i * ld + j;
        out[o] = act[o] > 0.0f ? v : 0.0f;
    }
};
struct AtomicAcc {  // out[i][j] += acc
    float* out;
    int ld;
    __device__ void operator()(int i, int j, float v) const { atomicAdd(&out[(size_t)i * ld + j], v); }
};

// ---- small kernels --------------------------------------------------------
// out[j] += sum_i a[i][j] for j < N <= 256: each block sums a slice of rows
// (thread t adds column t % N of rows t / N, t / N + 256 / N, ...; the rows
// are contiguous, so the loads coalesce), then one atomic per column.
__global__ void colsum_kernel(const float* __restrict__ a, int M, int N, int rows_per_block,
                              float* __restrict__ out) {
    __shared__ float part[256];
    const int t = threadIdx.x, lanes = blockDim.x / N * N;
    const int j = t % N, r0 = blockIdx.x * rows_per_block;
    const int r1 = min(M, r0 + rows_per_block);
    float s = 0.0f;
    if (t < lanes)
        for (int i = r0 + t / N; i < r1; i += lanes / N) s += a[(size_t)i * N + j];
    part[t] = t < lanes ? s : 0.0f;
    __syncthreads();
    if (t < N) {
        float tot = 0.0f;
        for (int k = t; k < lanes; k += N) tot += part[k];
        atomicAdd(&out[t], tot);
    }
}

void colsum(const float* a, int M, int N, float* out, cudaStream_t s) {
    if (M <= 0) return;
    const int rows = 64;  // short dependent-load chains per thread
    colsum_kernel<<<(M + rows - 1) / rows, 256, 0, s>>>(a, M, N, rows, out);
}

// ---- convolution weight gradients ------------------------------------------
// dW[c_out][tap][c_in] = sum over hits and positions p of
// bf16(dz[hit][p][c_out]) * bf16(act[hit][nbr(p, tap)][c_in]) (zero where the
// neighbour is outside the 5x5 grid), the operand rounding of the GEMMs.

// Position p of the 5x5 grid in the zero-bordered 7x7 grid; the neighbour at
// tap k is then a constant offset (k / 3 - 1) * 7 + k % 3 - 1.
__device__ __forceinline__ int pad7(int p) { return (p / 5 + 1) * 7 + p % 5 + 1; }

constexpr int WG_HB = 8;                        // hits per staged chunk
constexpr int WG_ROWS = WG_HB * 49;             // 392 padded positions
constexpr int WG_K = (WG_ROWS + 15) / 16 * 16;  // 400: whole k-steps
constexpr int WG_PAD = 8;                       // zero rows before and after (offsets -8..8)
constexpr int WG_ROW = WG_PAD + WG_K + WG_PAD;  // 416 bf16 of padded rows
constexpr int WG_LD = WG_ROW + 2;  // channel row pitch: 209 words (odd), so the 32
                                   // channels of one position land in 32 banks

// conv2: one warp per tap (9 warps), a 32 x 32 block of c_out x c_in each,
// on mma.sync m16n8k16; CTAs stride over chunks of WG_HB hits and add their
// sums to gw once.  Shared memory: dz and act transposed to
// [channel][padded position], bf16.
__global__ void __launch_bounds__(288) conv2_wgrad_kernel(const float* __restrict__ dz,
                                                          const float* __restrict__ act, int n,
                                                          float* __restrict__ gw) {
    extern __shared__ __align__(16) uint16_t wg_smem[];
    uint16_t* dzT = wg_smem;              // [C2][WG_LD]
    uint16_t* acT = wg_smem + C2 * WG_LD;  // [C1][WG_LD]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tq = lane & 3;
    const int tap = warp;
    const int off = (tap / 3 - 1) * 7 + tap % 3 - 1;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][b][c] = 0.0f;
    for (int i = tid; i < (C2 + C1) * WG_LD / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(wg_smem)[i] = 0u;  // borders and padding stay zero
    for (int h0 = blockIdx.x * WG_HB; h0 < n; h0 += gridDim.x * WG_HB) {
        __syncthreads();  // the previous chunk is read
        const int nh = min(WG_HB, n - h0);
        for (int e = tid; e < WG_HB * NPOS * 32; e += blockDim.x) {
            const int h = e / (NPOS * 32), pc = e - h * (NPOS * 32);
            const int pos = pc / 32, c = pc - pos * 32;
            const int row = WG_PAD + h * 49 + pad7(pos);
            const size_t src = ((size_t)(h0 + h) * NPOS + pos) * 32 + c;
            dzT[c * WG_LD + row] = h < nh ? bf16_bits(dz[src]) : (uint16_t)0;
            acT[c * WG_LD + row] = h < nh ? bf16_bits(act[src]) : (uint16_t)0;
        }
        __syncthreads();
        if (warp < 9) {
            for (int k0 = 0; k0 < WG_K; k0 += 16) {
                const int ka = WG_PAD + k0 + 2 * tq;
                uint32_t af[2][4], bfr[4][2];
#pragma unroll
                for (int mi = 0; mi < 2; mi++) {
                    const uint16_t* r0 = dzT + (mi * 16 + g) * WG_LD;
                    const uint16_t* r8 = r0 + 8 * WG_LD;
                    af[mi][0] = *reinterpret_cast<const uint32_t*>(r0 + ka);
                    af[mi][1] = *reinterpret_cast<const uint32_t*>(r8 + ka);
                    af[mi][2] = *reinterpret_cast<const uint32_t*>(r0 + ka + 8);
                    af[mi][3] = *reinterpret_cast<const uint32_t*>(r8 + ka + 8);
                }
#pragma unroll
                for (int ni = 0; ni < 4; ni++) {
                    const uint16_t* rb = acT + (ni * 8 + g) * WG_LD + ka + off;
                    bfr[ni][0] = (uint32_t)rb[0] | (uint32_t)rb[1] << 16;
                    bfr[ni][1] = (uint32_t)rb[8] | (uint32_t)rb[9] << 16;
                }
#pragma unroll
                for (int mi = 0; mi < 2; mi++)
#pragma unroll
                    for (int ni = 0; ni < 4; ni++) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
            }
        }
    }
    if (warp < 9) {
#pragma unroll
        for (int mi = 0; mi < 2; mi++)
#pragma unroll
            for (int ni = 0; ni < 4; ni++) {
                const int co = mi * 16 + g, ci = ni * 8 + 2 * tq;
                float* w0 = gw + (size_t)co * (9 * C1) + tap * C1 + ci;
                float* w8 = w0 + 8 * (9 * C1);
                atomicAdd(w0, acc[mi][ni][0]);
                atomicAdd(w0 + 1, acc[mi][ni][1]);
                atomicAdd(w8, acc[mi][ni][2]);
                atomicAdd(w8 + 1, acc[mi][ni][3]);
            }
    }
}

// conv1 (one input channel): thread t owns output (c_out = t / 9, tap = t % 9)
// and sums over its CTA's hits in float32 (bf16-rounded operands).
__global__ void __launch_bounds__(288) conv1_wgrad_kernel(const float* __restrict__ dz,
                                                          const float* __restrict__ x, int n,
                                                          float* __restrict__ gw) {
    __shared__ float sdz[WG_HB][NPOS][C1];
    __shared__ float sx[WG_HB][49];
    const int tid = threadIdx.x;
    const int co = tid / 9, tap = tid % 9;
    const int off = (tap / 3 - 1) * 7 + tap % 3 - 1;
    for (int i = tid; i < WG_HB * 49; i += blockDim.x) (&sx[0][0])[i] = 0.0f;
    float acc = 0.0f;
    for (int h0 = blockIdx.x * WG_HB; h0 < n; h0 += gridDim.x * WG_HB) {
        __syncthreads();
        const int nh = min(WG_HB, n - h0);
        for (int e = tid; e < WG_HB * NPOS * C1; e += blockDim.x) {
            const int h = e / (NPOS * C1);
            (&sdz[0][0][0])[e] =
                h < nh ? __bfloat162float(__float2bfloat16_rn(dz[(size_t)h0 * NPOS * C1 + e])) : 0.0f;
        }
        for (int e = tid; e < WG_HB * NPOS; e += blockDim.x) {
            const int h = e / NPOS, pos = e - h * NPOS;
            sx[h][pad7(pos)] =
                h < nh ? __bfloat162float(__float2bfloat16_rn(x[(size_t)h0 * NPOS + e])) : 0.0f;
        }
        __syncthreads();
        if (tid < C1 * 9)
            for (int h = 0; h < nh; h++)
#pragma unroll 5
                for (int pos = 0; pos < NPOS; pos++)
                    acc = __fmaf_rn(sdz[h][pos][co], sx[h][pad7(pos) + off], acc);
    }
    if (tid < C1 * 9) atomicAdd(&gw[co * 9 + tap], acc);
}

constexpr int C2_AP = 40;       // bf16 per input row in shared memory (32 used)
constexpr int C2_WS = 9 * 32 + 8;  // bf16 per weight row (288 used)
constexpr int C2_SMEM = (WG_ROW * C2_AP + 32 * C2_WS) * 2;

// conv2 forward (h2 = relu(conv(h1) + b2)) and the gradient of its input
// (dz1 = conv_transpose(dz2) where h1 > 0) on mma.sync m16n8k16: for tap k
// the input rows are the padded rows shifted by +off(k) (forward) or -off(k)
// (the transpose), so each is a GEMM over K = 9 taps x 32 channels from a
// zero-bordered [row][channel] tile of WG_HB hits.  8 warps; warp w computes
// the 16-row tiles w, w + 8, ... of the 400 padded rows, all 32 outputs.
template <bool DGRAD>
__global__ void __launch_bounds__(256) conv2_mma_kernel(const float* __restrict__ in,
                                                        const uint4* __restrict__ w2img,
                                                        const float* __restrict__ aux, int n,
                                                        float* __restrict__ out) {
    // input [padded row][channel] and weights [n][tap * 32 + k channel], rows
    // padded to 20 and 148 words so the fragment loads of 8 rows x 4 column
    // pairs fall in 32 distinct banks
    extern __shared__ __align__(16) uint16_t cm_smem[];
    uint16_t (*ap)[C2_AP] = reinterpret_cast<uint16_t (*)[C2_AP]>(cm_smem);
    uint16_t (*ws)[C2_WS] = reinterpret_cast<uint16_t (*)[C2_WS]>(cm_smem + WG_ROW * C2_AP);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tq = lane & 3;
    // weights, bf16 in this kernel's layout (w2_image_kernel), 16 bytes a load
    for (int e = tid; e < 32 * 9 * 32 / 8; e += blockDim.x) {
        const int a = e / (9 * 32 / 8), q = e - a * (9 * 32 / 8);
        *reinterpret_cast<uint4*>(&ws[a][8 * q]) = w2img[e];
    }
    for (int i = tid; i < WG_ROW * C2_AP / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(cm_smem)[i] = 0u;
    for (int h0 = blockIdx.x * WG_HB; h0 < n; h0 += gridDim.x * WG_HB) {
        __syncthreads();  // the previous chunk is read
        const int nh = min(WG_HB, n - h0);
        for (int e = tid; e < WG_HB * NPOS * 32; e += blockDim.x) {
            const int h = e / (NPOS * 32), pc = e - h * (NPOS * 32);
            const int pos = pc / 32, c = pc - pos * 32;
            ap[WG_PAD + h * 49 + pad7(pos)][c] =
                h < nh ? bf16_bits(in[(size_t)h0 * NPOS * 32 + e]) : (uint16_t)0;
        }
        __syncthreads();
        for (int mt = warp; mt < WG_K / 16; mt += 8) {
            float acc[4][4];
#pragma unroll
            for (int b = 0; b < 4; b++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[b][c] = 0.0f;
            const int r0 = mt * 16 + g;  // padded row of a0 / a2 (a1 / a3: r0 + 8)
#pragma unroll 3
            for (int tap = 0; tap < 9; tap++) {
                const int off = (tap / 3 - 1) * 7 + tap % 3 - 1;
                const int ra = WG_PAD + r0 + (DGRAD ? -off : off);
#pragma unroll
                for (int kc = 0; kc < 32; kc += 16) {
                    uint32_t af[4], bfr[4][2];
                    af[0] = *reinterpret_cast<const uint32_t*>(&ap[ra][kc + 2 * tq]);
                    af[1] = *reinterpret_cast<const uint32_t*>(&ap[ra + 8][kc + 2 * tq]);
                    af[2] = *reinterpret_cast<const uint32_t*>(&ap[ra][kc + 8 + 2 * tq]);
                    af[3] = *reinterpret_cast<const uint32_t*>(&ap[ra + 8][kc + 8 + 2 * tq]);
#pragma unroll
                    for (int ni = 0; ni < 4; ni++) {
                        const uint16_t* wb = &ws[ni * 8 + g][tap * 32 + kc + 2 * tq];
                        bfr[ni][0] = *reinterpret_cast<const uint32_t*>(wb);
                        bfr[ni][1] = *reinterpret_cast<const uint32_t*>(wb + 8);
                    }
#pragma unroll
                    for (int ni = 0; ni < 4; ni++) mma_bf16(acc[ni], af, bfr[ni]);
                }
            }
            // rows r0 and r0 + 8: outputs of interior positions of real hits
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int R = r0 + 8 * half, h = R / 49, pp = R - h * 49;
                const int y = pp / 7, x = pp - y * 7;
                if (h >= nh || y < 1 || y > 5 || x < 1 || x > 5) continue;
                const size_t o = ((size_t)(h0 + h) * NPOS + (y - 1) * 5 + (x - 1)) * 32;
#pragma unroll
                for (int ni = 0; ni < 4; ni++)
#pragma unroll
                    for (int j = 0; j < 2; j++) {
                        const int c = ni * 8 + 2 * tq + j;
                        const float v = acc[ni][2 * half + j];
                        if (DGRAD)
                            out[o + c] = aux[o + c] > 0.0f ? v : 0.0f;
                        else
                            out[o + c] = fmaxf(v + aux[c], 0.0f);
                    }
            }
        }
    }
}

// bf16 images of W2 for conv2_mma_kernel: [0, 9216) the forward layout
// [c_out][tap][c_in] (W2's own), [9216, 18432) the transpose [c_in][tap][c_out].
__global__ void w2_image_kernel(const float* __restrict__ w2, uint16_t* __restrict__ img) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 32 * 9 * 32) return;
    img[e] = bf16_bits(w2[e]);
    const int a = e / (9 * 32), rest = e - a * (9 * 32), tap = rest / 32, b = rest % 32;
    img[32 * 9 * 32 + e] = bf16_bits(w2[(size_t)b * (9 * C1) + tap * C1 + a]);
}

template <bool DGRAD>
cudaError_t launch_conv2_mma(const float* in, const uint16_t* w2img, const float* aux, int n,
                             float* out, cudaStream_t s) {
    static int attr_dev = -1;  // the shared-memory opt-in, once per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(conv2_mma_kernel<DGRAD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C2_SMEM);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const int grid = std::max(1, std::min(2 * 152, (n + WG_HB - 1) / WG_HB));
    conv2_mma_kernel<DGRAD><<<grid, 256, C2_SMEM, s>>>(in, reinterpret_cast<const uint4*>(w2img),
                                                        aux, n, out);
    return cudaGetLastError();
}

// a[i] = relu(a[i] + bias[i % N])
__global__ void bias_act_kernel(float* __restrict__ a, int total, int N,
                                const float* __restrict__ bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) a[i] = fmaxf(a[i] + bias[i % N], 0.0f);
}

// Softmax cross-entropy over out[:, 0:5] and masked squared error of
// out[:, 5:7]; dout and the loss (accumulated into *loss).
__global__ void loss_kernel(const float* __restrict__ out, const uint8_t* __restrict__ counts,
                            const float* __restrict__ tgt, const uint8_t* __restrict__ mask,
                            int B, float nreg, float lam, float* __restrict__ dout,
                            float* __restrict__ loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (b < B) {
        const float* o = out + (size_t)b * NOUT;
        float mx = o[0];
        for (int k = 1; k < 5; k++) mx = fmaxf(mx, o[k]);
        float e[5], s = 0.0f;
        for (int k = 0; k < 5; k++) {
            e[k] = expf(o[k] - mx);
            s += e[k];
        }
        const int n = min((int)counts[b], 4);
        float* d = dout + (size_t)b * NOUT;
        for (int k = 0; k < 5; k++) d[k] = (e[k] / s - (k == n ? 1.0f : 0.0f)) / (float)B;
        l = -logf(e[n] / s) / (float)B;
        const float m = mask[b] ? 1.0f : 0.0f;
        for (int k = 0; k < 2; k++) {
            const float diff = (o[5 + k] - tgt[(size_t)b * 2 + k]) * m;
            d[5 + k] = 2.0f * lam * diff / nreg;
            l += lam * diff * diff / nreg;
        }
    }
    for (int o2 = 16; o2; o2 >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o2);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// rows idx[i] of a training set into batch row i (one thread per float of a
// patch row, the labels by the row's first thread)
__global__ void take_kernel(const float* __restrict__ patches, const uint8_t* __restrict__ counts,
                            const float* __restrict__ targets, const uint8_t* __restrict__ mask,
                            const uint32_t* __restrict__ idx, uint32_t n,
                            float* __restrict__ p_out, uint8_t* __restrict__ c_out,
                            float* __restrict__ t_out, uint8_t* __restrict__ m_out) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * NPOS) return;
    const uint32_t i = (uint32_t)(t / NPOS), k = (uint32_t)(t % NPOS);
    const uint32_t j = idx[i];
    p_out[t] = patches[(size_t)j * NPOS + k];
    if (k == 0) {
        c_out[i] = counts[j];
        m_out[i] = mask[j];
        t_out[2 * (size_t)i] = targets[2 * (size_t)j];
        t_out[2 * (size_t)i + 1] = targets[2 * (size_t)j + 1];
    }
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ gr,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gv = gr[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gv;
    const float vi = b2 * v[i] + (1.0f - b2) * gv * gv;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// 5x5 patch of e / photon_kev around each hit's seed (zero outside the
// module): e recomputed exactly as the chain does, with the call's common
// mode of frame - frame_base (unit term, and for the stacked mean the module
// row and column terms).
template <bool MG>
__global__ void gather_kernel(pd::ChainParams p, const uint16_t* __restrict__ raw,
                              uint32_t frame_base, const float* __restrict__ cm,
                              const pd_hit* __restrict__ hits, uint32_t n,
                              float* __restrict__ patches, pd::MultiGain mg) {
    const uint32_t h = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (h >= n || lane >= NPOS) return;
    const pd_hit hit = hits[h];
    const uint32_t f = hit.frame - frame_base;
    const uint32_t m = hit.pixel / p.module_px, within = hit.pixel % p.module_px;
    const int r = (int)(within / p.cols) + lane / 5 - 2, c = (int)(within % p.cols) + lane % 5 - 2;
    float v = 0.0f;
    if (r >= 0 && r < (int)p.rows && c >= 0 && c < (int)p.cols) {
        const size_t g = (size_t)m * p.module_px + (size_t)r * p.cols + c;
        const uint32_t unit = m * p.units_per_module +
                              ((uint32_t)r / p.unit_rows) * p.units_per_row + (uint32_t)c / p.unit_cols;
        const float* cmf = cm + (size_t)f * cm_per_frame(p);
        float e;
        if (MG) {
            e = pd::mg_energy(mg, p.frame_px, raw[(size_t)f * p.frame_px + g], g, cmf[unit]);
        } else {
            const float d =
                __fsub_rn(__uint2float_rn(raw[(size_t)f * p.frame_px + g]), p.ped[g]);
            if (cm_kind(p) == PD_CM_MEAN_STACKED)
                e = pd::energy<true>(cm_after_gain(p), d, p.inv_gain[g], cmf[unit],
                                     cmf[p.units_per_frame + (size_t)m * p.rows + r],
                                     cmf[p.units_per_frame + (size_t)p.n_modules * p.rows +
                                         (size_t)m * p.cols + c]);
            else
                e = pd::energy<false>(cm_after_gain(p), d, p.inv_gain[g], cmf[unit], 0.0f, 0.0f);
        }
        v = __fdiv_rn(e, p.photon_kev);
    }
    patches[(size_t)h * NPOS + lane] = v;
}

// Replace count and (dx, dy) of hits the network is confident about; keep
// the classical values elsewhere.
__global__ void refine_kernel(const float* __restrict__ out, const pd_hit* __restrict__ in,
                              uint32_t n, float conf, float count_conf,
                              pd_hit* __restrict__ res) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    pd_hit h = in[b];
    const float* o = out + (size_t)b * NOUT;
    float mx = o[0];
    int arg = 0;
    for (int k = 1; k < 5; k++)
        if (o[k] > mx) {
            mx = o[k];
            arg = k;
        }
    float s = 0.0f;
    for (int k = 0; k < 5; k++) s += expf(o[k] - mx);
    const float pmax = 1.0f / s;
    if (pmax >= conf && arg >= 1) {
        if (pmax >= count_conf) h.count = (uint8_t)arg;
        h.dx = o[5];
        h.dy = o[6];
        h.flags |= PD_HIT_LEARNED;
    }
    res[b] = h;
}

int net_fail(int code, const std::string& why) { return pd::internal_fail(code, why.c_str()); }
int net_cuda(cudaError_t e, const char* what) {
    return net_fail(PD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

struct pd_net {
    uint32_t max_batch = 0;
    float *w = nullptr, *gw = nullptr, *m = nullptr, *v = nullptr;
    float *x0 = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *out = nullptr;
    float *dout = nullptr, *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;
    uint64_t step = 0;
    // tensor-core inference: bf16 weight image, bf16 h2, timeout flag
    uint8_t* tc_img = nullptr;
    uint16_t* tc_h2 = nullptr;
    uint16_t* w2img = nullptr;  // bf16 W2, forward and transposed (training)
    int* tc_err = nullptr;
};

namespace {

void free_net(pd_net* n) {
    if (!n) return;
    for (float* p : {n->w, n->gw, n->m, n->v, n->x0, n->h1, n->h2, n->h3, n->out, n->dout,
                     n->dz3, n->dz2, n->dz1})
        cudaFree(p);
    cudaFree(n->tc_img);
    cudaFree(n->tc_h2);
    cudaFree(n->w2img);
    cudaFree(n->tc_err);
    delete n;
}

// forward of n patches already in net->x0 (or at `x`) into net->out
cudaError_t forward(pd_net* net, const float* x, int n, cudaStream_t s) {
    const float* w = net->w;
    cudaError_t e;
    // conv1: [n*25, 9] x W1^T -> h1
    if ((e = gemm(n * NPOS, C1, 9, Im2col{x, 1}, ColMajor{w + OW1, 9},
                  BiasAct{net->h1, C1, w + OB1, true}, s)))
        return e;
    // conv2: [n*25, 288] x W2^T -> h2
    w2_image_kernel<<<(32 * 9 * 32 + 255) / 256, 256, 0, s>>>(w + OW2, net->w2img);
    if ((e = cudaGetLastError())) return e;
    if ((e = launch_conv2_mma<false>(net->h1, net->w2img, w + OB2, n, net->h2, s))) return e;
    // fc: [n, 800] x W3^T -> h3, split over K (8 slices summed atomically),
    // then the bias and ReLU
    if ((e = cudaMemsetAsync(net->h3, 0, (size_t)n * NH * sizeof(float), s))) return e;
    if ((e = gemm(n, NH, NPOS * C2, RowMajor{net->h2, NPOS * C2}, ColMajor{w + OW3, NPOS * C2},
                  AtomicAcc{net->h3, NH}, s, 8)))
        return e;
    bias_act_kernel<<<(n * NH + 255) / 256, 256, 0, s>>>(net->h3, n * NH, NH, w + OB3);
    if ((e = cudaGetLastError())) return e;
    // heads: [n, 64] x W4^T -> out
    return gemm(n, NOUT, NH, RowMajor{net->h3, NH}, ColMajor{w + OW4, NH},
                BiasAct{net->out, NOUT, w + OB4, false}, s);
}

// loss, dout and all parameter gradients (into net->gw, zeroed first)
cudaError_t backward(pd_net* net, const float* x, int n, const uint8_t* counts, const float* tgt,
                     const uint8_t* mask, float nreg, float lam, float* loss, cudaStream_t s) {
    const float* w = net->w;
    float* gw = net->gw;
    cudaError_t e;
    if ((e = cudaMemsetAsync(gw, 0, NPARAM * sizeof(float), s))) return e;
    loss_kernel<<<(n + 255) / 256, 256, 0, s>>>(net->out, counts, tgt, mask, n,
                                                std::max(1.0f, nreg), lam, net->dout, loss);
    if ((e = cudaGetLastError())) return e;
    // split-K of the fully connected layers' weight gradients (K = hits):
    // slices of about 64 hits, so each CTA runs two k-steps (these GEMMs
    // are small and bound by their load latency, not by the atomics)
    const int sp = std::max(1, std::min(64, n / 64));
    // heads
    if ((e = gemm(NOUT, NH, n, ColMajor{net->dout, NOUT}, RowMajor{net->h3, NH},
                  AtomicAcc{gw + OW4, NH}, s, sp)))
        return e;
    colsum(net->dout, n, NOUT, gw + OB4, s);
    if ((e = gemm(n, NH, NOUT, RowMajor{net->dout, NOUT}, RowMajor{w + OW4, NH},
                  ReluGrad{net->dz3, net->h3, NH}, s)))
        return e;
    // fc
    if ((e = gemm(NH, NPOS * C2, n, ColMajor{net->dz3, NH}, RowMajor{net->h2, NPOS * C2},
                  AtomicAcc{gw + OW3, NPOS * C2}, s, sp)))
        return e;
    colsum(net->dz3, n, NH, gw + OB3, s);
    if ((e = gemm(n, NPOS * C2, NH, RowMajor{net->dz3, NH}, RowMajor{w + OW3, NPOS * C2},
                  ReluGrad{net->dz2, net->h2, NPOS * C2}, s)))
        return e;
    // conv2: weights, bias, input
    {
        const int smem = (C2 + C1) * WG_LD * 2;
        static int attr_dev = -1;  // the shared-memory opt-in, once per device
        int dev = 0;
        cudaGetDevice(&dev);
        if (attr_dev != dev) {
            if ((e = cudaFuncSetAttribute(conv2_wgrad_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
                return e;
            attr_dev = dev;
        }
        const int grid = std::max(1, std::min(2 * 152, (n + WG_HB - 1) / WG_HB));
        conv2_wgrad_kernel<<<grid, 288, smem, s>>>(net->dz2, net->h1, n, gw + OW2);
        if ((e = cudaGetLastError())) return e;
    }
    colsum(net->dz2, n * NPOS, C2, gw + OB2, s);
    // (W2's images were built by the forward pass of the same step)
    if ((e = launch_conv2_mma<true>(net->dz2, net->w2img + 32 * 9 * 32, net->h1, n, net->dz1, s)))
        return e;
    // conv1: weights, bias
    {
        const int grid = std::max(1, std::min(2 * 152, (n + WG_HB - 1) / WG_HB));
        conv1_wgrad_kernel<<<grid, 288, 0, s>>>(net->dz1, x, n, gw + OW1);
        if ((e = cudaGetLastError())) return e;
    }
    colsum(net->dz1, n * NPOS, C1, gw + OB1, s);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

uint32_t pd_net_num_params(void) { return NPARAM; }

int pd_net_create(uint32_t max_batch, uint64_t seed, pd_net** out) {
    if (!out || !max_batch) return net_fail(PD_EINVAL, "pd_net_create: need out and max_batch");
    *out = nullptr;
    pd_net* n = new (std::nothrow) pd_net();
    if (!n) return net_fail(PD_ENOMEM, "host allocation failed");
    n->max_batch = max_batch;
    const size_t B = max_batch;
    struct { float** p; size_t count; } bufs[] = {
        {&n->w, NPARAM}, {&n->gw, NPARAM}, {&n->m, NPARAM}, {&n->v, NPARAM},
        {&n->x0, B * NPOS}, {&n->h1, B * NPOS * C1}, {&n->h2, B * NPOS * C2},
        {&n->h3, B * NH}, {&n->out, B * NOUT}, {&n->dout, B * NOUT}, {&n->dz3, B * NH},
        {&n->dz2, B * NPOS * C2}, {&n->dz1, B * NPOS * C1}};
    for (auto& b : bufs)
        if (cudaMalloc(b.p, b.count * sizeof(float)) != cudaSuccess) {
            free_net(n);
            return net_fail(PD_ENOMEM, "pd_net_create: device allocation failed");
        }
    if (cudaMalloc(&n->tc_img, pd::nettc::weight_image_bytes()) != cudaSuccess ||
        cudaMalloc(&n->tc_h2, pd::nettc::h2_bytes(max_batch)) != cudaSuccess ||
        cudaMalloc(&n->tc_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&n->w2img, 2 * 32 * 9 * 32 * sizeof(uint16_t)) != cudaSuccess ||
        cudaMemset(n->tc_err, 0, sizeof(int)) != cudaSuccess) {
        free_net(n);
        return net_fail(PD_ENOMEM, "pd_net_create: device allocation failed");
    }
    // weights and biases uniform in +-1/sqrt(fan_in), from a seeded generator
    std::vector<float> host(NPARAM, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int count, int fan_in) {
        const double b = 1.0 / std::sqrt((double)fan_in);
        std::uniform_real_distribution<double> ud(-b, b);
        for (int i = 0; i < count; i++) host[off + i] = (float)ud(rng);
    };
    fill(OW1, NW1, 9);
    fill(OB1, NB1, 9);
    fill(OW2, NW2, 9 * C1);
    fill(OB2, NB2, 9 * C1);
    fill(OW3, NW3, NPOS * C2);
    fill(OB3, NB3, NPOS * C2);
    fill(OW4, NW4, NH);
    fill(OB4, NB4, NH);
    if (cudaMemcpy(n->w, host.data(), NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->m, 0, NPARAM * 4) != cudaSuccess ||
        cudaMemset(n->v, 0, NPARAM * 4) != cudaSuccess) {
        free_net(n);
        return net_fail(PD_ECUDA, "pd_net_create: upload failed");
    }
    *out = n;
    return PD_OK;
}

int pd_net_set_params(pd_net* n, const float* host, uint32_t count) {
    if (!n || !host || count != NPARAM) return net_fail(PD_EINVAL, "pd_net_set_params: size");
    cudaError_t e = cudaMemcpy(n->w, host, NPARAM * 4, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? PD_OK : net_cuda(e, "pd_net_set_params");
}

int pd_net_get_params(pd_net* n, float* host, uint32_t count) {
    if (!n || !host || count != NPARAM) return net_fail(PD_EINVAL, "pd_net_get_params: size");
    cudaError_t e = cudaMemcpy(host, n->w, NPARAM * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PD_OK : net_cuda(e, "pd_net_get_params");
}

int pd_net_forward(pd_net* n, const float* patches, uint32_t count, float* out_dev, void* stream) {
    if (!n || (count && (!patches || !out_dev))) return net_fail(PD_EINVAL, "pd_net_forward: args");
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = pd::device_sm_count();
    for (uint32_t done = 0; done < count;) {
        const uint32_t b = std::min(n->max_batch, count - done);
        cudaError_t e = pd::nettc::forward(n->w, patches + (size_t)done * NPOS, b, n->tc_img,
                                           n->tc_h2, out_dev + (size_t)done * NOUT, n->tc_err,
                                           sms, s);
        if (e) return net_cuda(e, "pd_net_forward");
        done += b;
    }
    if (!count) return PD_OK;
    // a timed-out wait inside the kernels is reported here (this synchronises
    // the stream)
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return net_cuda(e, "pd_net_forward");
    if (flag) {
        cudaMemsetAsync(n->tc_err, 0, sizeof(int), s);
        return net_fail(PD_ETIMEDOUT, "pd_net_forward: tensor-core pipeline wait timed out");
    }
    return PD_OK;
}

int pd_net_gradients(pd_net* n, const float* patches, const uint8_t* counts, const float* targets,
                     const uint8_t* mask, uint32_t count, float n_reg, float lambda,
                     float* grads_dev, float* loss_dev, void* stream) {
    if (!n || !count || count > n->max_batch || !patches || !counts || !targets || !mask)
        return net_fail(PD_EINVAL, "pd_net_gradients: args (count <= max_batch)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = forward(n, patches, (int)count, s);
    if (!e) e = backward(n, patches, (int)count, counts, targets, mask, n_reg, lambda, loss_dev, s);
    if (!e && grads_dev)
        e = cudaMemcpyAsync(grads_dev, n->gw, NPARAM * 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PD_OK : net_cuda(e, "pd_net_gradients");
}

int pd_net_take(const float* patches, const uint8_t* counts, const float* targets,
                const uint8_t* mask, const uint32_t* idx, uint32_t count, float* p_out,
                uint8_t* c_out, float* t_out, uint8_t* m_out, void* stream) {
    if (!count) return PD_OK;
    if (!patches || !counts || !targets || !mask || !idx || !p_out || !c_out || !t_out || !m_out)
        return net_fail(PD_EINVAL, "pd_net_take: NULL argument");
    const uint64_t threads = (uint64_t)count * NPOS;
    take_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        patches, counts, targets, mask, idx, count, p_out, c_out, t_out, m_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PD_OK : net_cuda(e, "pd_net_take");
}

int pd_net_train_step(pd_net* n, const float* patches, const uint8_t* counts, const float* targets,
                      const uint8_t* mask, uint32_t count, float n_reg, float lambda, float lr,
                      float* loss_dev, void* stream) {
    int rc = pd_net_gradients(n, patches, counts, targets, mask, count, n_reg, lambda, nullptr,
                              loss_dev, stream);
    if (rc) return rc;
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)n->step);
    const float c2 = 1.0f - (float)std::pow(0.999, (double)n->step);
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n->w, n->gw, n->m, n->v,
                                                                        NPARAM, lr, b1, b2, c1, c2,
                                                                        1e-8f);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PD_OK : net_cuda(e, "adam");
}

int pd_net_refine(const float* out_dev, const pd_hit* hits_in, uint32_t count, float conf,
                  float count_conf, pd_hit* hits_out, void* stream) {
    if (count && (!out_dev || !hits_in || !hits_out)) return net_fail(PD_EINVAL, "pd_net_refine");
    if (!count) return PD_OK;
    refine_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        out_dev, hits_in, count, conf, count_conf, hits_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PD_OK : net_cuda(e, "refine");
}

void pd_net_destroy(pd_net* n) {
    if (!n) return;
    cudaDeviceSynchronize();
    free_net(n);
}

}  // extern "C"

namespace pd {
cudaError_t launch_gather(const ChainParams& p, const uint16_t* raw, uint32_t frame_base,
                          const float* cm, const pd_hit* hits, uint32_t n, float* patches,
                          cudaStream_t s, const MultiGain* mg) {
    if (!n) return cudaSuccess;
    const uint32_t per = 8;  // hits per 256-thread block (one warp each)
    const MultiGain m = mg ? *mg : MultiGain{};
    if (mg)
        gather_kernel<true><<<(n + per - 1) / per, 256, 0, s>>>(p, raw, frame_base, cm, hits, n,
                                                              patches, m);
    else
        gather_kernel<false><<<(n + per - 1) / per, 256, 0, s>>>(p, raw, frame_base, cm, hits, n,
                                                               patches, m);
    return cudaGetLastError();
}
}  // namespace pd
