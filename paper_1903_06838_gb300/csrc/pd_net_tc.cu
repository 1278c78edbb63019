// pd_net_tc.cu — inference of the learned count / offset network on the
// fifth-generation tensor cores: tcgen05.mma with bfloat16 operands staged in
// shared memory and float32 accumulators in tensor memory (TMEM).
//
// The network (conv3x3x32 -> conv3x3x32 -> FC64 -> 7 outputs on the 5x5
// neighbourhood of a seed) is the learned refinement the paper proposes as
// future work (abstract; sections "Methods", "Conclusions").  Numerics match
// the training path: every contraction multiplies bfloat16-rounded operands
// (weights, input patch, and the ReLU activations h1, h2, h3) and
// accumulates in float32; biases and ReLU are float32.
//
//   conv_kernel  one CTA holds 64 hits: their patches, all of h1 (64 x 25 x
//                32, bf16) and one 128-row im2col tile at a time.  conv1 and
//                conv2 are implicit GEMMs whose rows are (position, hit)
//                pairs: 13 tiles of 128 rows each (the last half full); a
//                conv2 tile is 18 MMAs of 128x32x16.  Accumulators alternate
//                between two 32-column TMEM buffers, so the epilogue of one
//                tile (bias, ReLU, bf16, store of h2) runs while the next
//                tile's MMAs execute.
//   fc_kernel    FC3 on 128 hits per CTA: h2 streams in 160-column chunks
//                (double-buffered) against W3 resident in shared memory;
//                the epilogue adds b3, applies ReLU and computes the 7 heads
//                (FC4) on the CUDA cores.
//
// Operand layout: the canonical no-swizzle K-major form: 8-row x 16-byte core
// matrices, core matrix (r, k) of a tile with R rows at byte
// ((k / 8) * (R / 8) + r / 8) * 128; descriptors carry the distance of
// K-adjacent core matrices (leading) and of row-adjacent ones (stride).
// Every wait on an mbarrier is bounded; a timeout sets an error flag.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pd_net_tc.cuh"

namespace pd {
namespace nettc {

namespace {

constexpr int NPOS = 25, C1 = 32, C2 = 32, NH = 64, NOUT = 7;
constexpr int K2 = 9 * C1;           // 288
constexpr int K3 = NPOS * C2;        // 800
constexpr int TB = 64;               // hits per conv tile
constexpr int TF = 128;              // hits per fc tile
constexpr int KCH = 160;             // fc K chunk
constexpr uint32_t kWaitLimit = 1u << 22;

// weight offsets (floats) in the parameter vector, as the training path
constexpr int OW1 = 0, OB1 = OW1 + C1 * 9, OW2 = OB1 + C1, OB2 = OW2 + C2 * K2, OW3 = OB2 + C2,
              OB3 = OW3 + NH * K3, OW4 = OB3 + NH, OB4 = OW4 + NOUT * NH;

// bf16 operand images of the weights (bytes)
constexpr uint32_t W1_BYTES = 32 * 16 * 2, W2_BYTES = 32 * K2 * 2, W3_BYTES = NH * K3 * 2;
constexpr uint32_t OFF_W1 = 0, OFF_W2 = OFF_W1 + W1_BYTES, OFF_W3 = OFF_W2 + W2_BYTES;

__host__ __device__ __forceinline__ uint32_t cm_off(uint32_t r, uint32_t k, uint32_t rows) {
    return ((k >> 3) * (rows >> 3) + (r >> 3)) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint16_t bf16_bits(float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&b);
}
__device__ __forceinline__ float bf16_round(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}
// kind::f16 instruction descriptor: f32 accumulate, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
// (volatile keeps tcgen05 operations in program order; shared-memory
// operands are published before the issue by fences and a barrier, so no
// memory clobber is needed and the issuing thread's table loads can run
// ahead)
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// bounded wait for the phase with parity `par`; false on timeout
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t par) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < kWaitLimit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(par)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 consecutive columns of this warp's 32 TMEM lanes, one wait
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// neighbour of position p at 3x3 offset k (k = 3 (dy + 1) + dx + 1), or -1
__device__ __forceinline__ int nb(int p, int k) {
    const int y = p / 5 + k / 3 - 1, x = p % 5 + k % 3 - 1;
    return (y >= 0 && y < 5 && x >= 0 && x < 5) ? y * 5 + x : -1;
}

// ---------------------------------------------------------------------------
// bf16 operand images of W1 (32 x 16, taps 9..15 zero), W2 (32 x 288) and
// W3 (64 x 800), K-major core-matrix layout, from the float32 parameters.
__global__ void prep_weights(const float* __restrict__ w, uint8_t* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 32 * 16) {
        const int r = i / 16, k = i % 16;
        *reinterpret_cast<uint16_t*>(img + OFF_W1 + cm_off(r, k, 32)) =
            bf16_bits(k < 9 ? w[OW1 + r * 9 + k] : 0.0f);
    }
    if (i < 32 * K2) {
        const int r = i / K2, k = i % K2;
        *reinterpret_cast<uint16_t*>(img + OFF_W2 + cm_off(r, k, 32)) = bf16_bits(w[OW2 + i]);
    }
    if (i < NH * K3) {
        const int r = i / K3, k = i % K3;
        *reinterpret_cast<uint16_t*>(img + OFF_W3 + cm_off(r, k, NH)) = bf16_bits(w[OW3 + i]);
    }
}

// ---------------------------------------------------------------------------
// conv1 + conv2 on tiles of 64 hits, h2 out as bf16 [n][800]; one CTA of 512
// threads per SM with specialised warps:
//   warps 0-7   conv1 on the CUDA cores (bf16 operands, float32 fused
//               multiply-adds) into one of two h1 stages: per position a
//               64-hit x 32-channel K-major block (4 KB), 100 KB per stage
//   warps 8-11  lane 0 of warp 8 + b issues the conv2 MMAs of the position
//               groups that use TMEM buffer b (128 columns, 4 positions):
//               an implicit GEMM read in place, the contribution of tap k to
//               position p being two 64x32x16 MMAs of h1 block nb(p, k)
//               against the W2 slice of tap k (taps outside the patch are not
//               issued).  One thread issues a small MMA about every 60
//               cycles; four issuing threads bring that to about 25.
//   warps 12-15 the epilogue: TMEM -> bias, ReLU, bf16 -> h2 (warp 12 + q
//               reads TMEM lanes 32q..32q+31)
// mbarriers hand the stages and TMEM buffers around (h1 full / empty, TMEM
// full / empty), so conv1 of the next tile, conv2 MMAs and the epilogue of
// earlier groups overlap.  Every wait is bounded; a timeout sets *err, stops
// every role, and the issuing lane waits (bounded) for its last commit
// before TMEM is freed.
constexpr int WS_PROD_WARPS = 8, WS_MMA_WARP0 = 8, WS_EPI_WARP0 = 12;
constexpr int WS_PROD = WS_PROD_WARPS * 32, WS_THREADS = 512;
constexpr uint32_t H1_STAGE = TB * NPOS * C1 * 2;  // 102 400 bytes
constexpr uint32_t WS_W2 = 0, WS_H1 = WS_W2 + W2_BYTES, WS_X = WS_H1 + 2 * H1_STAGE,
                   WS_W1 = WS_X + TB * NPOS * 2, WS_SMEM = WS_W1 + (9 * C1 + C1) * 4;
constexpr uint32_t kConvTmemCols = 512;
constexpr int kGroup = 4;     // conv2 positions per TMEM buffer
constexpr int kTBufs = 4;     // TMEM buffers of kGroup * 32 columns
constexpr int NG = (NPOS + kGroup - 1) / kGroup;
static_assert(WS_H1 % 128 == 0 && H1_STAGE % 128 == 0 && WS_W1 % 16 == 0, "alignment");
static_assert(kTBufs * kGroup * 32 <= (int)kConvTmemCols, "TMEM buffers");

__device__ __forceinline__ void bar_init_n(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(WS_PROD) : "memory");
}

__global__ void __launch_bounds__(WS_THREADS, 1)
    conv_kernel(const float* __restrict__ x, int n, const float* __restrict__ w,
                const uint8_t* __restrict__ img, uint16_t* __restrict__ h2, int* err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_prod_go;  // the producers' uniform decision for a tile
    __shared__ __align__(8) uint64_t s_h1_full[2], s_h1_empty[2], s_t_full[kTBufs],
        s_t_empty[kTBufs];
    __shared__ int s_nb[NPOS * 9];
    // per position: its valid (tap, channel half) MMAs as descriptor address
    // offsets (16-byte units): A block of the neighbour | W2 slice << 16
    __shared__ uint32_t s_mma[NPOS * 18];
    __shared__ int s_nmma[NPOS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint16_t* sx = reinterpret_cast<uint16_t*>(sm + WS_X);      // [64][25] bf16 patches
    float* w1t = reinterpret_cast<float*>(sm + WS_W1);           // [9][32] bf16-valued
    float* b1 = w1t + 9 * C1;                                    // [32]
    const uint32_t w2_addr = smem_u32(sm + WS_W2), h1_addr = smem_u32(sm + WS_H1);

    if (warp == 0) tmem_alloc(&s_tmem, kConvTmemCols);
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            bar_init_n(&s_h1_full[b], WS_PROD);
            bar_init_n(&s_h1_empty[b], kTBufs);  // one commit per issuing thread
        }
        for (int b = 0; b < kTBufs; b++) {
            bar_init_n(&s_t_full[b], 1);
            bar_init_n(&s_t_empty[b], 4);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < NPOS * 9; i += blockDim.x) s_nb[i] = nb(i / 9, i % 9);
    if (tid < NPOS) {
        int m = 0;
        for (int k = 0; k < 9; k++) {
            const int q = nb(tid, k);
            if (q < 0) continue;
            for (int kk = 0; kk < 2; kk++)
                s_mma[tid * 18 + m++] =
                    (uint32_t)((q * 4096 + kk * 2048) >> 4) |
                    ((uint32_t)(((4 * k + 2 * kk) * 512) >> 4) << 16);
        }
        s_nmma[tid] = m;
    }
    for (uint32_t i = tid; i < W2_BYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sm + WS_W2)[i] = reinterpret_cast<const uint4*>(img + OFF_W2)[i];
    for (int i = tid; i < 9 * C1; i += blockDim.x) {
        const int k = i / C1, c = i % C1;
        w1t[i] = bf16_round(w[OW1 + c * 9 + k]);
    }
    for (int i = tid; i < C1; i += blockDim.x) b1[i] = w[OB1 + i];
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    const int n_tiles = (n + TB - 1) / TB;
    // bounded wait that also gives up once another role has aborted
    auto wait_or_abort = [&](uint64_t* bar, uint32_t parity) -> bool {
        const uint32_t a = smem_u32(bar);
        for (uint32_t it = 0; it < kWaitLimit; it++) {
            uint32_t ok;
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                "selp.u32 %0, 1, 0, p;\n}"
                : "=r"(ok)
                : "r"(a), "r"(parity)
                : "memory");
            if (ok) return true;
            if ((it & 255) == 255 && s_abort) return false;
        }
        s_abort = 1;
        return false;
    };

    if (warp < WS_PROD_WARPS) {
        // ---- conv1 producers ------------------------------------------------
        const int ptid = tid;
        // B fragments of W1 (bf16, K = taps) and the biases of this lane's
        // channel pairs, for n-blocks of 8 channels
        uint32_t bw[4][2];
        float bias[4][2];
        {
            const int g = lane >> 2, tq = lane & 3;
            auto w1b = [&](int ch, int k) -> uint32_t {
                return k < 9 ? (uint32_t)bf16_bits(w[OW1 + ch * 9 + k]) : 0u;
            };
#pragma unroll
            for (int nb = 0; nb < 4; nb++) {
                const int ch = nb * 8 + g;
                bw[nb][0] = w1b(ch, 2 * tq) | (w1b(ch, 2 * tq + 1) << 16);
                bw[nb][1] = w1b(ch, 2 * tq + 8) | (w1b(ch, 2 * tq + 9) << 16);
                bias[nb][0] = w[OB1 + nb * 8 + 2 * tq];
                bias[nb][1] = w[OB1 + nb * 8 + 2 * tq + 1];
            }
        }
        // a tile's patches are loaded into registers one tile ahead, so the
        // global loads run during the previous tile's conv1
        constexpr int XPER = (TB * NPOS + WS_PROD - 1) / WS_PROD;
        float xn[XPER];
        auto load_x = [&](int t) {
            const int hit0 = t * TB, nh = t < n_tiles ? min(TB, n - hit0) : 0;
#pragma unroll
            for (int u = 0; u < XPER; u++) {
                const int e = ptid + u * WS_PROD;
                xn[u] = (e < TB * NPOS && e / NPOS < nh) ? x[(size_t)hit0 * NPOS + e] : 0.0f;
            }
        };
        load_x(blockIdx.x);
        int i = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, i++) {
            const int stage = i & 1;
            // one thread waits for the stage; every producer follows its
            // decision, so the named barriers below stay uniform
            if (ptid == 0)
                s_prod_go = wait_or_abort(&s_h1_empty[stage], ((i >> 1) & 1) ^ 1) && !s_abort;
            producers_sync();  // also: the previous tile's patches are no longer read
            if (!s_prod_go) break;
#pragma unroll
            for (int u = 0; u < XPER; u++) {
                const int e = ptid + u * WS_PROD;
                if (e < TB * NPOS) sx[e] = bf16_bits(xn[u]);
            }
            load_x(t + gridDim.x);
            producers_sync();
            uint8_t* h1 = sm + WS_H1 + stage * H1_STAGE;
            // conv1 as warp-level m16n8k16 MMAs: a 16-row block is 16 hits of
            // one position, K the 9 taps (7 zero columns), N 4 x 8 channels;
            // lane (g, t) gathers its A fragment from the patches: rows g and
            // g + 8, taps 2t, 2t + 1 and 2t + 8 (only t = 0 has tap 8)
            const int pwarp = warp, g = lane >> 2, tq = lane & 3;
            for (int rb = pwarp; rb < NPOS * (TB / 16); rb += WS_PROD_WARPS) {
                const int p = rb >> 2, h0 = (rb & 3) * 16;
                const int q0 = s_nb[p * 9 + 2 * tq], q1 = s_nb[p * 9 + 2 * tq + 1];
                const int q2 = tq == 0 ? s_nb[p * 9 + 8] : -1;
                const uint16_t* x0 = sx + (h0 + g) * NPOS;
                const uint16_t* x1 = x0 + 8 * NPOS;
                uint32_t a[4];
                a[0] = (q0 >= 0 ? (uint32_t)x0[q0] : 0u) | (q1 >= 0 ? (uint32_t)x0[q1] << 16 : 0u);
                a[1] = (q0 >= 0 ? (uint32_t)x1[q0] : 0u) | (q1 >= 0 ? (uint32_t)x1[q1] << 16 : 0u);
                a[2] = q2 >= 0 ? (uint32_t)x0[q2] : 0u;
                a[3] = q2 >= 0 ? (uint32_t)x1[q2] : 0u;
                uint8_t* blk = h1 + p * 4096;
#pragma unroll
                for (int nb = 0; nb < 4; nb++) {
                    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
                        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(bw[nb][0]),
                          "r"(bw[nb][1]));
                    const int ch = nb * 8 + 2 * tq;
                    const __nv_bfloat162 v0 = __float22bfloat162_rn(
                        make_float2(fmaxf(c[0] + bias[nb][0], 0.0f), fmaxf(c[1] + bias[nb][1], 0.0f)));
                    const __nv_bfloat162 v1 = __float22bfloat162_rn(
                        make_float2(fmaxf(c[2] + bias[nb][0], 0.0f), fmaxf(c[3] + bias[nb][1], 0.0f)));
                    *reinterpret_cast<__nv_bfloat162*>(blk + cm_off(h0 + g, ch, TB)) = v0;
                    *reinterpret_cast<__nv_bfloat162*>(blk + cm_off(h0 + g + 8, ch, TB)) = v1;
                }
            }
            fence_async_smem();  // h1 is read by the tensor cores
            bar_arrive(&s_h1_full[stage]);
        }
    } else if (warp < WS_EPI_WARP0) {
        // ---- conv2 MMA issue: lane 0 of warp 8 + b, TMEM buffer b -----------
        const int ib = warp - WS_MMA_WARP0;
        if (lane == 0) {
            const uint32_t id64 = idesc_bf16(64, 32);
            const uint64_t b_desc0 = sdesc(w2_addr, 512, 128);
            int i = 0, gq = 0;  // local tile, global group sequence
            bool issued = false;
            uint64_t* last = nullptr;
            uint32_t last_par = 0;
            for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, i++) {
                const int stage = i & 1;
                if (!wait_or_abort(&s_h1_full[stage], (i >> 1) & 1)) break;
                fence_after();
                const uint64_t a_desc0 = sdesc(h1_addr + stage * H1_STAGE, 1024, 128);
                bool ok = true;
                for (int g = 0; g < NG; g++, gq++) {
                    const int b = gq % kTBufs;
                    if (b != ib) continue;  // another thread's buffer
                    if (!wait_or_abort(&s_t_empty[b], ((gq / kTBufs) & 1) ^ 1)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    for (int pi = 0; pi < kGroup; pi++) {
                        const int p = g * kGroup + pi;
                        if (p >= NPOS) break;
                        const uint32_t d = tmem + (uint32_t)((b * kGroup + pi) * 32);
                        const int nm = s_nmma[p];
                        const uint32_t* tab = s_mma + p * 18;
                        for (int e = 0; e < nm; e++) {
                            const uint32_t o = tab[e];
                            mma(d, a_desc0 + (o & 0xFFFFu), b_desc0 + (o >> 16), id64, e);
                        }
                    }
                    commit(&s_t_full[b]);
                    issued = true;
                    last = &s_t_full[b];
                    last_par = (gq / kTBufs) & 1;
                }
                if (!ok) break;
                commit(&s_h1_empty[stage]);  // stage free once these MMAs complete
            }
            if (s_abort) {
                atomicExch(err, 1);
                if (issued) wait_bar(last, last_par);  // bounded
            }
        }
        __syncwarp();
    } else if (warp >= WS_EPI_WARP0) {
        // ---- conv2 epilogue (warps 8-11, TMEM lane quadrant q) ---------------
        const int q = warp - WS_EPI_WARP0;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int qhit = q * 16 + lane;  // M = 64: row r in TMEM lane (r / 16) * 32 + r % 16
        float b2[C2];
#pragma unroll
        for (int c = 0; c < C2; c++) b2[c] = w[OB2 + c];
        int gq = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            const int hit0 = t * TB, nh = min(TB, n - hit0);
            bool ok = true;
            for (int g = 0; g < NG; g++, gq++) {
                const int b = gq % kTBufs;
                // lane 0 waits and the warp follows it (tcgen05.ld is warp-wide)
                const int got = __shfl_sync(
                    0xffffffffu, lane == 0 ? (int)wait_or_abort(&s_t_full[b], (gq / kTBufs) & 1) : 0,
                    0);
                if (!got) {
                    ok = false;
                    break;
                }
                fence_after();
                for (int pi = 0; pi < kGroup; pi++) {
                    const int p = g * kGroup + pi;
                    if (p >= NPOS) break;
                    uint32_t r[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)((b * kGroup + pi) * 32), r);
                    if (lane < 16 && qhit < nh) {
                        uint32_t pk[16];
#pragma unroll
                        for (int c = 0; c < 32; c += 2) {
                            const float2 z = __fadd2_rn(
                                make_float2(__uint_as_float(r[c]), __uint_as_float(r[c + 1])),
                                make_float2(b2[c], b2[c + 1]));
                            const __nv_bfloat162 v =
                                __float22bfloat162_rn(make_float2(fmaxf(z.x, 0.0f), fmaxf(z.y, 0.0f)));
                            pk[c / 2] = *reinterpret_cast<const uint32_t*>(&v);
                        }
                        uint4* dst = reinterpret_cast<uint4*>(h2 + (size_t)(hit0 + qhit) * K3 +
                                                              p * C2);
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            dst[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2],
                                                pk[4 * j + 3]);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(&s_t_empty[b]);
            }
            if (!ok) break;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (s_abort && tid == 0) atomicExch(err, 1);
    if (warp == 0) tmem_free(tmem, kConvTmemCols);
}

// ---------------------------------------------------------------------------
// FC3 + heads on tiles of 128 hits.
constexpr uint32_t FC_W3 = 0, FC_A = FC_W3 + W3_BYTES, FC_ABUF = TF * KCH * 2,
                   FC_PART = FC_A + 2 * FC_ABUF, FC_SMEM = FC_PART + 128 * 8 * 4;
static_assert(FC_A % 128 == 0, "alignment");

__global__ void __launch_bounds__(256, 1)
    fc_kernel(const uint16_t* __restrict__ h2, int n, const float* __restrict__ w,
              const uint8_t* __restrict__ img, float* __restrict__ out, int* err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ float s_w4[NOUT * NH];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* part = reinterpret_cast<float*>(sm + FC_PART);  // [128][8]
    const uint32_t w3_addr = smem_u32(sm + FC_W3);

    if (warp == 0) tmem_alloc(&s_tmem, 64);
    if (tid == 0)
        for (int b = 0; b < 2; b++) bar_init(&s_bar[b]);
    for (uint32_t i = tid; i < W3_BYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sm + FC_W3)[i] = reinterpret_cast<const uint4*>(img + OFF_W3)[i];
    for (int i = tid; i < NOUT * NH; i += blockDim.x) s_w4[i] = bf16_round(w[OW4 + i]);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    uint32_t par[2] = {0, 0};
    bool pend[2] = {false, false};
    bool ok = true;
    auto waitp = [&](int b) -> bool {
        const bool r = __syncthreads_and(wait_bar(&s_bar[b], par[b]));
        if (r) {
            par[b] ^= 1;
            pend[b] = false;
        }
        return r;
    };
    const uint32_t id3 = idesc_bf16(128, NH);
    const int n_tiles = (n + TF - 1) / TF;
    const int half = warp >> 2;
    const int erow = (warp & 3) * 32 + lane;

    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int hit0 = t * TF, nh = min(TF, n - hit0);
        constexpr int NCH = K3 / KCH;  // 5 chunks of 10 MMAs
        // chunk c of this tile into buffer c & 1 by asynchronous 16-byte
        // copies (rows past the last hit are zero-filled)
        auto load_chunk = [&](int c) {
            const uint32_t abuf = smem_u32(sm + FC_A + (c & 1) * FC_ABUF);
            for (int e = tid; e < TF * (KCH / 8); e += blockDim.x) {
                const int r = e / (KCH / 8), kc = (e % (KCH / 8)) * 8;
                const bool in = r < nh;
                const uint16_t* src = h2 + (size_t)(hit0 + (in ? r : 0)) * K3 + c * KCH + kc;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                                 abuf + cm_off(r, kc, TF)),
                             "l"(src), "r"(in ? 16 : 0)
                             : "memory");
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        load_chunk(0);
        for (int c = 0; c < NCH && ok; c++) {
            const int buf = c & 1;
            if (c + 1 < NCH) {
                if (c >= 1) {  // buffer (c + 1) & 1 was read by the MMAs of chunk c - 1
                    ok = waitp((c + 1) & 1);
                    if (!ok) break;
                }
                load_chunk(c + 1);
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // chunk c landed
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            }
            fence_async_smem();
            fence_before();
            __syncthreads();
            fence_after();
            if (tid == 0) {
                const uint32_t a0 = smem_u32(sm + FC_A + buf * FC_ABUF);
                for (int s = 0; s < KCH / 16; s++) {
                    const int ks = c * (KCH / 16) + s;  // global K step
                    mma(tmem, sdesc(a0 + s * 2 * (TF / 8) * 128, (TF / 8) * 128, 128),
                        sdesc(w3_addr + ks * 2 * (NH / 8) * 128, (NH / 8) * 128, 128), id3,
                        (c > 0 || s > 0) ? 1u : 0u);
                }
                commit(&s_bar[buf]);
            }
            pend[buf] = true;
        }
        if (!ok) {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            break;
        }
        // the last two chunks (buffers 1 and 0)
        for (int c = NCH - 2; c < NCH && ok; c++) ok = waitp(c & 1);
        if (!ok) break;
        fence_after();
        // epilogue: h3 = relu(acc + b3) rounded to bf16, heads on the CUDA
        // cores; warps 4..7 take columns 32..63 and pass partial sums
        uint32_t ra[16], rb[16];
        const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16) + half * 32;
        tmem_ld16(tbase, ra);
        tmem_ld16(tbase + 16, rb);
        float acc[NOUT];
#pragma unroll
        for (int o = 0; o < NOUT; o++) acc[o] = 0.0f;
#pragma unroll
        for (int c = 0; c < 32; c++) {
            const int ch = half * 32 + c;
            const float z = __uint_as_float(c < 16 ? ra[c] : rb[c - 16]) + w[OB3 + ch];
            const float h = bf16_round(fmaxf(z, 0.0f));
#pragma unroll
            for (int o = 0; o < NOUT; o++) acc[o] = __fmaf_rn(h, s_w4[o * NH + ch], acc[o]);
        }
        if (half == 1)
#pragma unroll
            for (int o = 0; o < NOUT; o++) part[erow * 8 + o] = acc[o];
        fence_before();
        __syncthreads();
        if (half == 0 && erow < nh)
#pragma unroll
            for (int o = 0; o < NOUT; o++)
                out[(size_t)(hit0 + erow) * NOUT + o] = acc[o] + part[erow * 8 + o] + w[OB4 + o];
        __syncthreads();  // partial sums, A buffers and TMEM reused by the next tile
    }
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        for (int b = 0; b < 2; b++)
            if (pend[b]) wait_bar(&s_bar[b], par[b]);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_free(tmem, 64);
}

}  // namespace

size_t weight_image_bytes() { return OFF_W3 + W3_BYTES; }
size_t h2_bytes(uint32_t max_batch) { return (size_t)max_batch * K3 * 2; }

cudaError_t forward(const float* w, const float* x, uint32_t n, uint8_t* img, uint16_t* h2,
                    float* out, int* err, int sms, cudaStream_t s) {
    if (!n) return cudaSuccess;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(conv_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, WS_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     FC_SMEM);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    prep_weights<<<(NH * K3 + 255) / 256, 256, 0, s>>>(w, img);
    const int conv_tiles = (int)((n + TB - 1) / TB), fc_tiles = (int)((n + TF - 1) / TF);
    conv_kernel<<<std::min(conv_tiles, sms), WS_THREADS, WS_SMEM, s>>>(x, (int)n, w, img, h2, err);
    fc_kernel<<<std::min(fc_tiles, sms), 256, FC_SMEM, s>>>(h2, (int)n, w, img, out, err);
    return cudaGetLastError();
}

}  // namespace nettc
}  // namespace pd
