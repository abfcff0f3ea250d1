// Plane-proposal network: 6 layers of 3x3 convolutions (32 channels, ReLU
// between layers) on (left RGB, right RGB, disparity) at quarter resolution,
// predicting (d, a, b) per quarter-resolution pixel; bilinear upsampling turns
// the prediction into a full-resolution map of plane labels that the
// expansion kernel can draw candidates from.
//
// Convolutions are implicit GEMMs on the tensor cores (BF16 operands, FP32
// accumulation):
//   forward      Y[p][o]   = sum_k Xpatch[p][k] W[k][o]        (M = 128 positions, N = Cout, K = 9 Cin)
//                on tcgen05.mma with the accumulator in tensor memory; the input
//                band is staged by the bulk-copy engine and each tap's A operand
//                is that band seen from a shifted shared-memory descriptor
//   input grad   dX        = the same kernel with flipped, transposed weights
//   weight grad  dW^T[k][o] = sum_p Xpatch[p][k] dZ[p][o]     (M = 9 Cin, N = Cout, K = pixels)
//                on tcgen05.mma: each CTA accumulates its pixel range in tensor
//                memory and writes a partial sum; a second kernel adds the
//                partials in a fixed order, so gradients are bit-reproducible
// Activations live on a zero-padded grid (see Geo below): BF16 in 8-channel
// blocks, channels padded to a multiple of 16; the weights have an FP32 master
// copy updated by Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lem.h"
#include "lem_internal.h"

namespace lemcnn {

constexpr int kLayers = 6;
// padded input / output channels of each layer (the real ones: 7/32 ... 32/3)
constexpr int kCin[kLayers] = {16, 32, 32, 32, 32, 32};
constexpr int kCout[kLayers] = {32, 32, 32, 32, 32, 16};
constexpr int kRealCin[kLayers] = {7, 32, 32, 32, 32, 32};
constexpr int kRealCout[kLayers] = {32, 32, 32, 32, 32, 3};
constexpr int kTileP = 128;  // pixels per CTA

// element index of (row, k) in a rows x K bf16 matrix stored in the K-major
// no-swizzle core-matrix layout (8 rows x 8 elements = 128 contiguous bytes per
// core matrix, core matrix (row / 8, k / 8) at (row / 8 * K / 8 + k / 8) * 64):
// the weights are kept in global memory in this order, so one bulk copy makes
// the tensor cores' B operand
__host__ __device__ __forceinline__ size_t cm_index(int row, int k, int K) {
    return ((size_t)(row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// tcgen05 (5th-generation tensor core) helpers.  Operands sit in shared memory
// in the no-swizzle K-major canonical layout: 8-row x 16-byte core matrices,
// each 128 contiguous bytes; core matrix (row group g, k chunk c) of a tile
// with K columns is at byte (g * K/8 + c) * 128.  The accumulator lives in
// tensor memory (TMEM): row i of the 128-row tile is TMEM lane i.
// ---------------------------------------------------------------------------
__device__ unsigned int g_mma_timeouts = 0;  // waits on an MMA completion that gave up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// shared-memory matrix descriptor: start address, leading-dimension byte offset
// (between core matrices along K), stride byte offset (between 8-row groups),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// bounded wait for phase 0 of an mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait0(uint32_t mbar, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar)
            : "memory");
        if (done) return true;
    }
    return false;
}
// bounded wait for the phase of parity `parity` of an mbarrier; false if it gave up
__device__ __forceinline__ bool mbar_wait_parity(uint32_t mbar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
template <int N>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&out)[N]);
template <>
__device__ __forceinline__ void tmem_load_row<32>(uint32_t taddr, float (&o)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) o[j] = __uint_as_float(r[j]);
}
template <>
__device__ __forceinline__ void tmem_load_row<16>(uint32_t taddr, float (&o)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j] = __uint_as_float(r[j]);
}

constexpr int kConvThreads = 128;       // 4 warps: warp w reads TMEM lanes 32w .. 32w + 31
constexpr int kMmaWaitLimit = 1 << 22;  // try_wait polls before a wait gives up
static_assert(kConvThreads == kTileP, "one thread per pixel row of the tile");

// ---------------------------------------------------------------------------
// Activation layout.  B images of H x W pixels sit in one zero-padded grid:
// each image gets a zero row above and below and a zero column left and right,
// so a pixel's 3x3 neighbourhood is the positions q + dy (W + 2) + dx around
// its position q, and the images follow one another row after row.  G guard
// positions before and after the grid keep every shifted read in the buffer.
//   bf16 tensors (layer inputs, output gradients): channel-blocked, 8 channels
//     (16 bytes) per position and block, block c8 of position q at
//     (c8 * Ptot + q) * 8 elements;
//   fp32 tensors (pre-activations, input gradients): C values per position at
//     q * C.
// Only interior positions are ever written; the rest stay zero (the buffers
// are cleared whenever the geometry changes).
// ---------------------------------------------------------------------------
struct Geo {
    int B, H, W;    // images and their size
    int Wp;         // W + 2
    int64_t G;      // guard positions before the grid (= Wp + 1)
    int64_t P;      // positions of the grid, B (H + 2) Wp
    int64_t tiles;  // 128-position tiles covering the grid
    int64_t Ptot;   // G + 128 tiles + G
};
inline Geo make_geo(int B, int H, int W) {
    Geo g;
    g.B = B;
    g.H = H;
    g.W = W;
    g.Wp = W + 2;
    g.G = g.Wp + 1;
    g.P = (int64_t)B * (H + 2) * g.Wp;
    g.tiles = (g.P + 127) / 128;
    g.Ptot = g.G + 128 * g.tiles + g.G;
    return g;
}
// position of interior pixel p (0 .. B H W - 1, images one after the other, row-major)
__host__ __device__ __forceinline__ int64_t pos_of(const Geo &g, int64_t p) {
    const int64_t x = p % g.W, r = p / g.W;  // r: row over all images
    const int64_t b = r / g.H, y = r - b * g.H;
    return g.G + (b * (g.H + 2) + y + 1) * g.Wp + x + 1;
}
// whether grid position q holds a pixel (not padding or guard)
__device__ __forceinline__ bool interior(const Geo &g, int64_t q) {
    const int64_t t = q - g.G;
    if (t < 0 || t >= g.P) return false;
    const int64_t r = t / g.Wp, x = t - r * g.Wp;
    const int64_t y = r % (g.H + 2);
    return x >= 1 && x <= g.W && y >= 1 && y <= g.H;
}

// Y = conv3x3(X) (+ bias) as an implicit GEMM on the tensor cores, 128 grid
// positions per CTA (M = 128, N = COUT, K = 9 CIN), with no patch gathering:
// one thread copies, per 8-channel block, the positions q0 - G .. q0 + 127 + G
// of X into shared memory with the bulk-copy engine (cp.async.bulk, completion
// on an mbarrier); each block's run of 16-byte positions is a column of 8-row
// core matrices of the K-major no-swizzle layout, so the A operand of tap
// (dy, dx) is the same shared memory seen from an offset of dy (W + 2) + dx
// positions.  The weights (B, COUT x 9CIN), kept in global memory in that
// layout, come with the same copies; one thread issues the 9 CIN / 16
// tcgen05.mma into a TMEM accumulator and each
// warp reads its 32 rows back for the epilogue, which writes interior
// positions only.
//   X  : bf16, channel-blocked (CIN / 8 blocks);  Bt : COUT x (9 CIN) bf16 (row o holds W[k][o]) in the
//        core-matrix order of cm_index;
//   Z  : optional fp32 pre-activation, COUT per position;  Y : optional bf16 output, channel-blocked
//        (ReLU if relu)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_conv(const bf16 *X, Geo g, const bf16 *Bt, const float *bias,
                                                       float *Z, bf16 *Y, int relu) {
    constexpr int K = 9 * CIN, KC = K / 8, CH = CIN / 8;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    const int span = 128 + 2 * (int)g.G;                   // positions staged per block
    const uint32_t SA = ((uint32_t)span * 16u + 127u) & ~127u;  // bytes per block in shared memory
    unsigned char *Bs = sm_raw;                            // COUT x K, core-matrix layout
    unsigned char *As = sm_raw + (size_t)COUT * K * 2;     // CH blocks of SA bytes
    __shared__ __align__(8) uint64_t mbar_ld, mbar_mma;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q0 = g.G + (int64_t)blockIdx.x * kTileP;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        // bulk copies of the weights (already in core-matrix order) and of the CH
        // blocks: positions q0 - G .. q0 + 127 + G (16 bytes each)
        const uint32_t bytes = (uint32_t)span * 16u, wbytes = (uint32_t)(COUT * K * 2);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(&mbar_ld)),
                     "r"(bytes * CH + wbytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                smem_u32(Bs)),
            "l"(Bt), "r"(wbytes), "r"(smem_u32(&mbar_ld))
            : "memory");
        for (int c = 0; c < CH; ++c) {
            const bf16 *src = X + ((size_t)c * g.Ptot + (size_t)(q0 - g.G)) * 8;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    smem_u32(As + (size_t)c * SA)),
                "l"(src), "r"(bytes), "r"(smem_u32(&mbar_ld))
                : "memory");
        }
    }
    __shared__ float s_bias[COUT];
    if (tid < COUT) s_bias[tid] = bias ? bias[tid] : 0.f;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = tmem_base;
    __shared__ int s_ok;
    if (tid == 0) {
        s_ok = mbar_wait0(smem_u32(&mbar_ld), kMmaWaitLimit) ? 1 : 0;
        if (s_ok) {
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            constexpr uint32_t idesc = idesc_bf16(kTileP, COUT);
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const int shift = (t / 3 - 1) * g.Wp + (t % 3 - 1);
                const uint32_t at = a0 + (uint32_t)((int)g.G + shift) * 16u;
#pragma unroll 1
                for (int j = 0; j < CH / 2; ++j) {
                    // K step: channels 16j .. 16j + 15 of tap t = blocks 2j, 2j + 1
                    const uint64_t ad = smem_desc(at + (uint32_t)(2 * j) * SA, SA, 128);
                    const uint64_t bd = smem_desc(b0 + (uint32_t)(t * (CH / 2) + j) * 256, 128, KC * 128);
                    mma_tc(tbase, ad, bd, idesc, (t > 0 || j > 0) ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar_mma))
                         : "memory");
        } else {
            atomicAdd(&g_mma_timeouts, 1u);
            // the copies may still be in flight: one more bounded wait before the
            // CTA's shared memory can be handed on
            mbar_wait0(smem_u32(&mbar_ld), kMmaWaitLimit);
        }
    }
    __syncthreads();
    const bool ok = s_ok && mbar_wait0(smem_u32(&mbar_mma), kMmaWaitLimit);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        float acc[COUT];
        tmem_load_row<COUT>(tbase + ((uint32_t)(warp * 32) << 16), acc);
        const int64_t q = q0 + warp * 32 + lane;
        if (interior(g, q)) {
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] += s_bias[o];
            if (Z) {
                float4 *z4 = reinterpret_cast<float4 *>(Z + (size_t)q * COUT);
#pragma unroll
                for (int o = 0; o < COUT; o += 4) z4[o / 4] = make_float4(acc[o], acc[o + 1], acc[o + 2], acc[o + 3]);
            }
            if (Y) {
#pragma unroll
                for (int o = 0; o < COUT; o += 8) {
                    __nv_bfloat162 h[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float x0 = relu ? fmaxf(acc[o + 2 * j], 0.f) : acc[o + 2 * j];
                        const float x1 = relu ? fmaxf(acc[o + 2 * j + 1], 0.f) : acc[o + 2 * j + 1];
                        h[j] = __floats2bfloat162_rn(x0, x1);
                    }
                    *reinterpret_cast<uint4 *>(Y + ((size_t)(o / 8) * g.Ptot + (size_t)q) * 8) =
                        *reinterpret_cast<uint4 *>(h);
                }
            }
        }
    } else if (tid == 0 && s_ok) {
        atomicAdd(&g_mma_timeouts, 1u);
        // give the MMAs in flight one more bounded chance before TMEM is freed
        mbar_wait0(smem_u32(&mbar_mma), kMmaWaitLimit);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;\n" ::"r"(tbase));
}

// Weight gradient on the tensor cores: dW^T[k][o] = sum_p Xpatch[p][k] dZ[p][o]
// as a GEMM with M = 9 CIN (padded to 128-row tiles), N = COUT and K = the
// pixels.  Each CTA takes `tiles_per_cta` consecutive 128-pixel tiles; per tile
// the patches (A, MP x 128 pixels) and dZ (B, COUT x 128 pixels) are written to
// shared memory in the K-major core-matrix layout, and one thread issues the
// MMAs of every M tile into the CTA's accumulator in tensor memory (accumulating
// across the tiles).  The CTA then writes its partial dW (COUT x 9CIN, the
// layout of gW) and bias partial (sum of dZ over its pixels, in pixel order) to
// part / partb at its index; k_wgrad_reduce adds the partials in index order.
// The pixels are the interior pixels of the grid in order; a patch reads the
// zero padding beyond its image's border.
//   X  : bf16, channel-blocked (CIN / 8 blocks);  dZ : bf16, channel-blocked (COUT / 8 blocks)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_wgrad_tc(const bf16 *X, const bf16 *dZ, Geo g, int tiles_per_cta,
                                                           float *part, float *partb) {
    constexpr int K = 9 * CIN, MT = (K + 127) / 128, MP = MT * 128, PC = kTileP / 8, CH = CIN / 8;
    constexpr int TC = MT * COUT <= 32 ? 32 : (MT * COUT <= 64 ? 64 : (MT * COUT <= 128 ? 128 : 256));
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *As = sm_raw;                             // MP x 128 pixels
    unsigned char *Bs = sm_raw + (size_t)MP * kTileP * 2;   // COUT x 128 pixels
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float s_db[COUT];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = g.H * g.W * g.B;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (tid < COUT) s_db[tid] = 0.f;
    // rows K .. MP of A are padding: zero once, never written again
    for (int q = tid; q < (MP - K) * PC; q += kConvThreads) {
        const int m = K + q / PC, c = q % PC;
        *reinterpret_cast<uint4 *>(As + ((size_t)(m >> 3) * PC + c) * 128 + (m & 7) * 16) = make_uint4(0, 0, 0, 0);
    }
    bool ok = true;
    int issued = 0;
    for (int t = 0; t < tiles_per_cta; ++t) {
        const int p0 = (blockIdx.x * tiles_per_cta + t) * kTileP;
        if (p0 >= n) break;
        // the MMAs of the previous tile read A and B: wait for them before refilling
        if (issued > 0) ok = ok && mbar_wait_parity(smem_u32(&mbar), (uint32_t)((issued - 1) & 1), kMmaWaitLimit);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        {
            // thread r: pixel r of the tile; its patch values are column r of A,
            // its output gradient column r of B
            const int r = tid, p = p0 + r;
            const int64_t q = p < n ? pos_of(g, p) : 0;  // neighbours outside the image read zero padding
            for (int c = 0; c < 9 * CH; ++c) {
                const int tap = c / CH, c8 = c - tap * CH;
                const int64_t qs = q + (tap / 3 - 1) * g.Wp + (tap % 3 - 1);
                uint4 val = make_uint4(0, 0, 0, 0);
                if (p < n) val = *reinterpret_cast<const uint4 *>(X + ((size_t)c8 * g.Ptot + (size_t)qs) * 8);
                const bf16 *e = reinterpret_cast<const bf16 *>(&val);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int m = tap * CIN + c8 * 8 + j;
                    *reinterpret_cast<bf16 *>(As + ((size_t)(m >> 3) * PC + (r >> 3)) * 128 + (m & 7) * 16 +
                                              (r & 7) * 2) = e[j];
                }
            }
#pragma unroll
            for (int c8 = 0; c8 < COUT / 8; ++c8) {
                uint4 val = make_uint4(0, 0, 0, 0);
                if (p < n) val = *reinterpret_cast<const uint4 *>(dZ + ((size_t)c8 * g.Ptot + (size_t)q) * 8);
                const bf16 *e = reinterpret_cast<const bf16 *>(&val);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int o = c8 * 8 + j;
                    *reinterpret_cast<bf16 *>(Bs + ((size_t)(o >> 3) * PC + (r >> 3)) * 128 + (o & 7) * 16 +
                                              (r & 7) * 2) = e[j];
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // bias partial: the tile's dZ summed in pixel order
        if (tid < COUT) {
            float sb = 0.f;
            for (int r = 0; r < kTileP; ++r)
                sb += __bfloat162float(*reinterpret_cast<const bf16 *>(
                    Bs + ((size_t)(tid >> 3) * PC + (r >> 3)) * 128 + (tid & 7) * 16 + (r & 7) * 2));
            s_db[tid] += sb;
        }
        if (tid == 0) {
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            constexpr uint32_t idesc = idesc_bf16(128, COUT);
#pragma unroll 1
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll 1
                for (int kk = 0; kk < kTileP / 16; ++kk) {
                    const uint64_t ad = smem_desc(a0 + mt * 16 * PC * 128 + kk * 256, 128, PC * 128);
                    const uint64_t bd = smem_desc(b0 + kk * 256, 128, PC * 128);
                    mma_tc(tmem_base + (uint32_t)(mt * COUT), ad, bd, idesc, (issued > 0 || kk > 0) ? 1u : 0u);
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar))
                         : "memory");
        }
        ++issued;
        // (the bias sums above read B before the next tile overwrites it)
        __syncthreads();
    }
    if (issued > 0) ok = ok && mbar_wait_parity(smem_u32(&mbar), (uint32_t)((issued - 1) & 1), kMmaWaitLimit);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float *pw = part + (size_t)blockIdx.x * COUT * K;
    if (issued > 0 && ok) {
#pragma unroll 1
        for (int mt = 0; mt < MT; ++mt) {
            float acc[COUT];
            tmem_load_row<COUT>(tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * COUT), acc);
            const int m = mt * 128 + warp * 32 + lane;
            if (m < K)
#pragma unroll
                for (int o = 0; o < COUT; ++o) pw[(size_t)o * K + m] = acc[o];
        }
    } else {
        // no tile, or a wait that gave up: this partial is zero
        if (!ok && tid == 0) atomicAdd(&g_mma_timeouts, 1u);
        if (!ok && tid == 0) mbar_wait_parity(smem_u32(&mbar), (uint32_t)((issued - 1) & 1), kMmaWaitLimit);
        for (int q = tid; q < COUT * K; q += kConvThreads) pw[q] = 0.f;
    }
    if (tid < COUT) partb[(size_t)blockIdx.x * COUT + tid] = s_db[tid];
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base), "r"(TC));
}

// gW += sum over the G partials (in index order), gB likewise
__global__ void k_wgrad_reduce(const float *part, const float *partb, int G, int KK, int COUT, float *gW, float *gB) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < KK) {
        float s = 0.f;
        for (int g = 0; g < G; ++g) s += part[(size_t)g * KK + i];
        gW[i] += s;
    } else if (i < KK + COUT) {
        const int o = i - KK;
        float s = 0.f;
        for (int g = 0; g < G; ++g) s += partb[(size_t)g * COUT + o];
        gB[o] += s;
    }
}

// dZprev = dX * (Zprev > 0) as bf16 (ReLU backward) at every position of the
// grid (zero where Zprev is: padding and guards); dX, Zprev fp32 with C values
// per position, dZ channel-blocked
__global__ void k_relu_back(const float *dX, const float *Zprev, int C, int64_t Ptot, bf16 *dZ) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ptot * C) return;
    const int64_t q = i / C;
    const int c = (int)(i - q * C);
    dZ[((size_t)(c >> 3) * Ptot + (size_t)q) * 8 + (c & 7)] = __float2bfloat16_rn(Zprev[i] > 0.f ? dX[i] : 0.f);
}

// L1 loss on (d, a, b) over the n interior pixels: out holds 16 fp32 values
// per grid position (channels 0..2 used), target 3 per pixel; writes d loss /
// d out (bf16, two channel blocks, padded channels zero) and accumulates the loss
__global__ void k_l1_loss(const float *out, const float *target, Geo g, int n, float s0, float s1, float s2,
                          float inv_n, bf16 *dout, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (p < n) {
        const float sc[3] = {s0, s1, s2};
        const int64_t q = pos_of(g, p);
        for (int c = 0; c < 16; ++c) {
            float gval = 0.f;
            if (c < 3) {
                const float diff = out[(size_t)q * 16 + c] - target[(size_t)p * 3 + c];
                l += sc[c] * fabsf(diff);
                gval = (diff > 0.f ? sc[c] : (diff < 0.f ? -sc[c] : 0.f)) * inv_n;
            }
            dout[((size_t)(c >> 3) * g.Ptot + (size_t)q) * 8 + (c & 7)] = __float2bfloat16_rn(gval);
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l * inv_n);
}

// Adam on the fp32 master weights of one layer (real channels only), then the
// bf16 copies: forward Bt[o][k] and input-gradient Bf[c][k'] (flipped taps,
// roles of channels swapped), both in the core-matrix order of cm_index.
//   w: (3,3,Cin,Cout) real sizes, fp32;  gW: dW in the padded GEMM layout COUT x 9CIN
__global__ void k_adam(float *w, float *m, float *v, const float *gW, int ci, int co, int CIN, int COUT, float lr,
                       float b1, float b2, float eps, float c1, float c2, bf16 *Bt, bf16 *Bf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 9 * ci * co) return;
    const int o = idx % co, c = (idx / co) % ci, tap = idx / (co * ci);
    const float gr = gW[(size_t)o * 9 * CIN + tap * CIN + c];
    const float mm = b1 * m[idx] + (1.f - b1) * gr;
    const float vv = b2 * v[idx] + (1.f - b2) * gr * gr;
    m[idx] = mm;
    v[idx] = vv;
    const float wn = w[idx] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    w[idx] = wn;
    Bt[cm_index(o, tap * CIN + c, 9 * CIN)] = __float2bfloat16_rn(wn);
    if (Bf) Bf[cm_index(c, (8 - tap) * COUT + o, 9 * COUT)] = __float2bfloat16_rn(wn);
}

__global__ void k_adam_bias(float *b, float *m, float *v, const float *g, int co, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int o = threadIdx.x;
    if (o >= co) return;
    const float mm = b1 * m[o] + (1.f - b1) * g[o];
    const float vv = b2 * v[o] + (1.f - b2) * g[o] * g[o];
    m[o] = mm;
    v[o] = vv;
    b[o] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// bf16 copies of all layers from the fp32 master weights
__global__ void k_pack_weights(const float *w, int ci, int co, int CIN, int COUT, bf16 *Bt, bf16 *Bf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 9 * ci * co) return;
    const int o = idx % co, c = (idx / co) % ci, tap = idx / (co * ci);
    Bt[cm_index(o, tap * CIN + c, 9 * CIN)] = __float2bfloat16_rn(w[idx]);
    if (Bf) Bf[cm_index(c, (8 - tap) * COUT + o, 9 * COUT)] = __float2bfloat16_rn(w[idx]);
}

// quarter-resolution input: x (fp32, 7 values per pixel: R,G,B of left, R,G,B
// of right /255, disparity / dmax) of the n interior pixels -> bf16, two
// channel blocks (channels 7..15 zero)
__global__ void k_pack_input(const float *x, Geo g, int n, bf16 *X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * 16) return;
    const int p = i / 16, c = i % 16;
    const int64_t q = pos_of(g, p);
    X[((size_t)(c >> 3) * g.Ptot + (size_t)q) * 8 + (c & 7)] = __float2bfloat16_rn(c < 7 ? x[(size_t)p * 7 + c] : 0.f);
}

// network output (pre-activation of the last layer, 16 values per grid
// position) -> y (3 channels per interior pixel)
__global__ void k_take3(const float *z, Geo g, int n, float *y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * 3) return;
    y[i] = z[(size_t)pos_of(g, i / 3) * 16 + i % 3];
}

// shared memory of k_conv: the weights and CIN / 8 blocks of 128 + 2 G positions;
// at most 226 KB of the 227 KB a CTA may have, the rest for its static shared
// variables (grids up to 1597 columns)
constexpr size_t kConvSmemMax = 226 * 1024;
template <int CIN, int COUT>
size_t conv_smem(const Geo &g) {
    const size_t SA = ((size_t)(128 + 2 * g.G) * 16 + 127) & ~(size_t)127;
    return (size_t)2 * 9 * CIN * COUT + (size_t)(CIN / 8) * SA;
}
constexpr int kWgParts = 148;  // most CTAs (partial sums) of one weight-gradient launch

template <int CIN, int COUT>
size_t wgrad_smem() {
    return (size_t)2 * kTileP * ((9 * CIN + 127) / 128 * 128 + COUT);
}

template <int CIN, int COUT>
cudaError_t conv(const bf16 *X, const Geo &g, const bf16 *Bt, const float *bias, float *Z, bf16 *Y, int relu,
                 cudaStream_t st) {
    const size_t sm = conv_smem<CIN, COUT>(g);
    if (sm > kConvSmemMax) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_conv<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_conv<CIN, COUT><<<(unsigned)g.tiles, kConvThreads, sm, st>>>(X, g, Bt, bias, Z, Y, relu);
    return cudaGetLastError();
}

// part: kWgParts * COUT * 9CIN floats, partb: kWgParts * COUT floats (scratch)
template <int CIN, int COUT>
cudaError_t wgrad(const bf16 *X, const bf16 *dZ, const Geo &g, float *dW, float *dB, float *part, float *partb,
                  cudaStream_t st) {
    const size_t sm = wgrad_smem<CIN, COUT>();
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int tiles = (g.H * g.W * g.B + kTileP - 1) / kTileP;
    const int per = (tiles + kWgParts - 1) / kWgParts;
    const int G = (tiles + per - 1) / per;
    k_wgrad_tc<CIN, COUT><<<G, kConvThreads, sm, st>>>(X, dZ, g, per, part, partb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int KK = COUT * 9 * CIN;
    k_wgrad_reduce<<<(KK + COUT + 255) / 256, 256, 0, st>>>(part, partb, G, KK, COUT, dW, dB);
    return cudaGetLastError();
}

}  // namespace lemcnn

using namespace lemcnn;

struct lem_cnn {
    cudaStream_t st = nullptr;
    float *w[kLayers] = {}, *b[kLayers] = {};     // fp32 master weights (3,3,ci,co), bias
    float *mw[kLayers] = {}, *vw[kLayers] = {}, *mb[kLayers] = {}, *vb[kLayers] = {};
    bf16 *Bt[kLayers] = {}, *Bf[kLayers] = {};    // forward / input-gradient GEMM layouts
    float *gW[kLayers] = {}, *gB[kLayers] = {};   // gradients (padded GEMM layout)
    float *wpart = nullptr, *wpartb = nullptr;    // per-CTA partials of the weight gradient
    // activations on the zero-padded grid of the current geometry (all images
    // of a training step), for up to cap grid positions
    int64_t cap = 0;
    int geoB = 0, geoH = 0, geoW = 0;             // geometry the buffers were last cleared for
    bf16 *act[kLayers] = {};                      // layer inputs (bf16, channel-blocked), act[0] = packed input
    float *pre[kLayers] = {};                     // pre-activations (fp32, Cout per position)
    bf16 *dz = nullptr;                           // d loss / d pre-activation (bf16, 32 ch, channel-blocked)
    float *dx = nullptr;                          // d loss / d layer input (fp32, 32 per position)
    float *loss = nullptr;
    int step = 0;
    std::string err;
};

namespace {
thread_local std::string g_cnn_err;

int cnn_fail(lem_cnn *net, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e);
    if (net) net->err = m;
    g_cnn_err = m;
    return e == cudaErrorMemoryAllocation ? LEM_ERR_OOM : LEM_ERR_CUDA;
}
#define CNN_CUDA(net, call)                                          \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cnn_fail((net), e_, #call);    \
    } while (0)

size_t nweights(int l) { return (size_t)9 * kRealCin[l] * kRealCout[l]; }

// Buffers for the grid of B images of H x W: allocated for at least its
// positions, and cleared whenever the geometry changes, so that every padding
// and guard position reads zero (the kernels write interior positions only).
int ensure_geometry(lem_cnn *net, const Geo &g) {
    if (g.Ptot > net->cap) {
        // pointers are cleared as they are freed, so a failed allocation below
        // leaves nothing dangling for a later call or lem_cnn_destroy
        auto drop = [](auto *&p) {
            cudaFree(p);
            p = nullptr;
        };
        net->cap = 0;
        net->geoB = net->geoH = net->geoW = 0;
        for (int l = 0; l < kLayers; ++l) drop(net->act[l]);
        for (int l = 0; l < kLayers; ++l) drop(net->pre[l]);
        drop(net->dz);
        drop(net->dx);
        for (int l = 0; l < kLayers; ++l) CNN_CUDA(net, cudaMalloc(&net->act[l], sizeof(bf16) * g.Ptot * kCin[l]));
        for (int l = 0; l < kLayers; ++l) CNN_CUDA(net, cudaMalloc(&net->pre[l], sizeof(float) * g.Ptot * kCout[l]));
        CNN_CUDA(net, cudaMalloc(&net->dz, sizeof(bf16) * g.Ptot * 32));
        CNN_CUDA(net, cudaMalloc(&net->dx, sizeof(float) * g.Ptot * 32));
        net->cap = g.Ptot;
    }
    if (net->geoB != g.B || net->geoH != g.H || net->geoW != g.W) {
        for (int l = 0; l < kLayers; ++l) {
            CNN_CUDA(net, cudaMemsetAsync(net->act[l], 0, sizeof(bf16) * g.Ptot * kCin[l], net->st));
            CNN_CUDA(net, cudaMemsetAsync(net->pre[l], 0, sizeof(float) * g.Ptot * kCout[l], net->st));
        }
        CNN_CUDA(net, cudaMemsetAsync(net->dz, 0, sizeof(bf16) * g.Ptot * 32, net->st));
        CNN_CUDA(net, cudaMemsetAsync(net->dx, 0, sizeof(float) * g.Ptot * 32, net->st));
        net->geoB = g.B;
        net->geoH = g.H;
        net->geoW = g.W;
    }
    return LEM_OK;
}

cudaError_t forward(lem_cnn *net, const Geo &g) {
    cudaStream_t st = net->st;
    cudaError_t e = conv<16, 32>(net->act[0], g, net->Bt[0], net->b[0], net->pre[0], net->act[1], 1, st);
    for (int l = 1; l < 5 && e == cudaSuccess; ++l)
        e = conv<32, 32>(net->act[l], g, net->Bt[l], net->b[l], net->pre[l], net->act[l + 1], 1, st);
    if (e == cudaSuccess) e = conv<32, 16>(net->act[5], g, net->Bt[5], net->b[5], net->pre[5], nullptr, 0, st);
    return e;
}

// backward over the grid from d loss / d output (in net->dz, 16 channels);
// accumulates into gW / gB
cudaError_t backward(lem_cnn *net, const Geo &g) {
    cudaStream_t st = net->st;
    cudaError_t e = cudaSuccess;
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
        // weight gradient of layer l: input act[l], output gradient dz
        if (l == 5) e = wgrad<32, 16>(net->act[5], net->dz, g, net->gW[5], net->gB[5], net->wpart, net->wpartb, st);
        else if (l == 0) e = wgrad<16, 32>(net->act[0], net->dz, g, net->gW[0], net->gB[0], net->wpart, net->wpartb, st);
        else e = wgrad<32, 32>(net->act[l], net->dz, g, net->gW[l], net->gB[l], net->wpart, net->wpartb, st);
        if (e != cudaSuccess || l == 0) break;
        // input gradient: conv of dz with the flipped, transposed weights
        if (l == 5) e = conv<16, 32>(net->dz, g, net->Bf[5], nullptr, net->dx, nullptr, 0, st);
        else e = conv<32, 32>(net->dz, g, net->Bf[l], nullptr, net->dx, nullptr, 0, st);
        if (e != cudaSuccess) break;
        // ReLU of layer l-1, over every grid position (padding stays zero)
        const int C = kCout[l - 1];
        const int64_t cnt = g.Ptot * C;
        k_relu_back<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(net->dx, net->pre[l - 1], C, g.Ptot, net->dz);
        e = cudaGetLastError();
    }
    return e;
}
}  // namespace

namespace {
// reports (and clears) tensor-core completion waits that gave up
int check_mma_timeouts(lem_cnn *net) {
    unsigned int t = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&t, g_mma_timeouts, sizeof(t));
    if (e != cudaSuccess) return cnn_fail(net, e, "reading the MMA timeout counter");
    if (t) {
        const unsigned int zero = 0;
        cudaMemcpyToSymbol(g_mma_timeouts, &zero, sizeof(zero));
        const std::string m = std::to_string(t) + " convolution tile(s) gave up waiting for the tensor core";
        if (net) net->err = m;
        g_cnn_err = m;
        return LEM_ERR_CUDA;
    }
    return LEM_OK;
}
}  // namespace

extern "C" {

const char *lem_cnn_last_error(const lem_cnn *net) { return net ? net->err.c_str() : g_cnn_err.c_str(); }

int lem_cnn_check(lem_cnn *net) {
    if (!net) return LEM_ERR_ARG;
    CNN_CUDA(net, cudaStreamSynchronize(net->st));
    return check_mma_timeouts(net);
}

int lem_cnn_create(uint64_t seed, void *stream, lem_cnn **out) {
    if (!out) return LEM_ERR_ARG;
    *out = nullptr;
    lem_cnn *net = new lem_cnn();
    net->st = (cudaStream_t)stream;
    auto bail = [&](int rc) {
        lem_cnn_destroy(net);
        return rc;
    };
    // He initialisation from a fixed generator (host), zero biases
    uint64_t s = seed ^ 0x2545F4914F6CDD1Dull;
    auto uni = [&]() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1.0p-53;
    };
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = nweights(l);
        std::vector<float> hw(nw);
        const double sd = std::sqrt(2.0 / (9.0 * kRealCin[l])) * (l == kLayers - 1 ? 0.1 : 1.0);
        for (size_t i = 0; i < nw; ++i) {
            // Box-Muller normal
            const double u1 = std::max(uni(), 1e-300), u2 = uni();
            hw[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
        cudaError_t e = cudaMalloc(&net->w[l], sizeof(float) * nw);
        if (e == cudaSuccess) e = cudaMemcpy(net->w[l], hw.data(), sizeof(float) * nw, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&net->b[l], sizeof(float) * kCout[l]);
        if (e == cudaSuccess) e = cudaMemset(net->b[l], 0, sizeof(float) * kCout[l]);
        for (float **p : {&net->mw[l], &net->vw[l]})
            if (e == cudaSuccess) {
                e = cudaMalloc(p, sizeof(float) * nw);
                if (e == cudaSuccess) e = cudaMemset(*p, 0, sizeof(float) * nw);
            }
        for (float **p : {&net->mb[l], &net->vb[l], &net->gB[l]})
            if (e == cudaSuccess) {
                e = cudaMalloc(p, sizeof(float) * kCout[l]);
                if (e == cudaSuccess) e = cudaMemset(*p, 0, sizeof(float) * kCout[l]);
            }
        const size_t gemm = (size_t)kCout[l] * 9 * kCin[l];
        if (e == cudaSuccess) e = cudaMalloc(&net->Bt[l], sizeof(bf16) * gemm);
        if (e == cudaSuccess) e = cudaMemset(net->Bt[l], 0, sizeof(bf16) * gemm);
        if (e == cudaSuccess) e = cudaMalloc(&net->Bf[l], sizeof(bf16) * gemm);
        if (e == cudaSuccess) e = cudaMemset(net->Bf[l], 0, sizeof(bf16) * gemm);
        if (e == cudaSuccess) e = cudaMalloc(&net->gW[l], sizeof(float) * gemm);
        if (e == cudaSuccess) e = cudaMemset(net->gW[l], 0, sizeof(float) * gemm);
        if (e == cudaSuccess) {
            k_pack_weights<<<(int)((nw + 255) / 256), 256, 0, net->st>>>(net->w[l], kRealCin[l], kRealCout[l],
                                                                        kCin[l], kCout[l], net->Bt[l], net->Bf[l]);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return bail(cnn_fail(net, e, "lem_cnn_create"));
    }
    cudaError_t e = cudaMalloc(&net->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->wpart, sizeof(float) * kWgParts * 32 * 9 * 32);
    if (e == cudaSuccess) e = cudaMalloc(&net->wpartb, sizeof(float) * kWgParts * 32);
    if (e != cudaSuccess) return bail(cnn_fail(net, e, "lem_cnn_create"));
    *out = net;
    return LEM_OK;
}

int lem_cnn_destroy(lem_cnn *net) {
    if (!net) return LEM_OK;
    for (int l = 0; l < kLayers; ++l) {
        for (float *p : {net->w[l], net->b[l], net->mw[l], net->vw[l], net->mb[l], net->vb[l], net->gW[l], net->gB[l],
                         net->pre[l]})
            cudaFree(p);
        cudaFree(net->Bt[l]);
        cudaFree(net->Bf[l]);
    }
    for (int l = 0; l < kLayers; ++l) cudaFree(net->act[l]);
    cudaFree(net->dz);
    cudaFree(net->dx);
    cudaFree(net->loss);
    cudaFree(net->wpart);
    cudaFree(net->wpartb);
    delete net;
    return LEM_OK;
}

int64_t lem_cnn_num_params(void) {
    int64_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (int64_t)nweights(l) + kRealCout[l];
    return n;
}

int lem_cnn_get_params(lem_cnn *net, float *host) {
    if (!net || !host) return LEM_ERR_ARG;
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        CNN_CUDA(net, cudaMemcpy(host + o, net->w[l], sizeof(float) * nweights(l), cudaMemcpyDeviceToHost));
        o += nweights(l);
        CNN_CUDA(net, cudaMemcpy(host + o, net->b[l], sizeof(float) * kRealCout[l], cudaMemcpyDeviceToHost));
        o += kRealCout[l];
    }
    return LEM_OK;
}

int lem_cnn_set_params(lem_cnn *net, const float *host) {
    if (!net || !host) return LEM_ERR_ARG;
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        CNN_CUDA(net, cudaMemcpy(net->w[l], host + o, sizeof(float) * nweights(l), cudaMemcpyHostToDevice));
        o += nweights(l);
        CNN_CUDA(net, cudaMemcpy(net->b[l], host + o, sizeof(float) * kRealCout[l], cudaMemcpyHostToDevice));
        o += kRealCout[l];
        const size_t nw = nweights(l);
        k_pack_weights<<<(int)((nw + 255) / 256), 256, 0, net->st>>>(net->w[l], kRealCin[l], kRealCout[l], kCin[l],
                                                                    kCout[l], net->Bt[l], net->Bf[l]);
        CNN_CUDA(net, cudaGetLastError());
    }
    return LEM_OK;
}

int lem_cnn_forward(lem_cnn *net, const float *x, int H4, int W4, float *out) {
    if (!net || !x || !out || H4 < 1 || W4 < 1) return LEM_ERR_ARG;
    const Geo g = make_geo(1, H4, W4);
    if (conv_smem<32, 32>(g) > kConvSmemMax || g.Ptot * 32 > (int64_t)INT32_MAX) return LEM_ERR_ARG;
    const size_t n = (size_t)H4 * W4;
    int rc = ensure_geometry(net, g);
    if (rc != LEM_OK) return rc;
    k_pack_input<<<(int)((n * 16 + 255) / 256), 256, 0, net->st>>>(x, g, (int)n, net->act[0]);
    CNN_CUDA(net, cudaGetLastError());
    CNN_CUDA(net, forward(net, g));
    k_take3<<<(int)((n * 3 + 255) / 256), 256, 0, net->st>>>(net->pre[5], g, (int)n, out);
    CNN_CUDA(net, cudaGetLastError());
    return LEM_OK;
}

int lem_cnn_gradients(lem_cnn *net, const float *x, const float *target, int n_images, int H4, int W4,
                      const float *scale, float *loss, float *grads) {
    if (!net || !x || !target || n_images < 1 || H4 < 1 || W4 < 1 || !scale) return LEM_ERR_ARG;
    // all images go through each layer in one launch: the batch is one grid of
    // n_images zero-padded images whose 3x3 neighbourhoods stop at each image's border
    const Geo g = make_geo(n_images, H4, W4);
    const size_t n = (size_t)H4 * W4 * n_images;
    if (conv_smem<32, 32>(g) > kConvSmemMax || g.Ptot * 32 > (int64_t)INT32_MAX || n * 16 > (size_t)INT32_MAX)
        return LEM_ERR_ARG;
    int rc = ensure_geometry(net, g);
    if (rc != LEM_OK) return rc;
    for (int l = 0; l < kLayers; ++l) {
        CNN_CUDA(net, cudaMemsetAsync(net->gW[l], 0, sizeof(float) * kCout[l] * 9 * kCin[l], net->st));
        CNN_CUDA(net, cudaMemsetAsync(net->gB[l], 0, sizeof(float) * kCout[l], net->st));
    }
    CNN_CUDA(net, cudaMemsetAsync(net->loss, 0, sizeof(float), net->st));
    const float inv_n = 1.f / (float)n;
    k_pack_input<<<(int)((n * 16 + 255) / 256), 256, 0, net->st>>>(x, g, (int)n, net->act[0]);
    CNN_CUDA(net, cudaGetLastError());
    CNN_CUDA(net, forward(net, g));
    k_l1_loss<<<(int)((n + 255) / 256), 256, 0, net->st>>>(net->pre[5], target, g, (int)n, scale[0], scale[1],
                                                         scale[2], inv_n, net->dz, net->loss);
    CNN_CUDA(net, cudaGetLastError());
    CNN_CUDA(net, backward(net, g));
    if (loss) CNN_CUDA(net, cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, net->st));
    if (grads) {
        // real-channel gradients in the (3,3,ci,co) + bias order of lem_cnn_get_params
        std::vector<float> g;
        for (int l = 0; l < kLayers; ++l) {
            std::vector<float> gw((size_t)kCout[l] * 9 * kCin[l]), gb(kCout[l]);
            CNN_CUDA(net, cudaMemcpyAsync(gw.data(), net->gW[l], sizeof(float) * gw.size(), cudaMemcpyDeviceToHost,
                                          net->st));
            CNN_CUDA(net, cudaMemcpyAsync(gb.data(), net->gB[l], sizeof(float) * gb.size(), cudaMemcpyDeviceToHost,
                                          net->st));
            CNN_CUDA(net, cudaStreamSynchronize(net->st));
            for (int tap = 0; tap < 9; ++tap)
                for (int c = 0; c < kRealCin[l]; ++c)
                    for (int o = 0; o < kRealCout[l]; ++o) g.push_back(gw[(size_t)o * 9 * kCin[l] + tap * kCin[l] + c]);
            for (int o = 0; o < kRealCout[l]; ++o) g.push_back(gb[o]);
        }
        std::copy(g.begin(), g.end(), grads);
    }
    CNN_CUDA(net, cudaStreamSynchronize(net->st));
    return check_mma_timeouts(net);
}

int lem_cnn_train_step(lem_cnn *net, const float *x, const float *target, int n_images, int H4, int W4,
                       const float *scale, float lr, float *loss) {
    int rc = lem_cnn_gradients(net, x, target, n_images, H4, W4, scale, loss, nullptr);
    if (rc != LEM_OK) return rc;
    ++net->step;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = nweights(l);
        k_adam<<<(int)((nw + 255) / 256), 256, 0, net->st>>>(net->w[l], net->mw[l], net->vw[l], net->gW[l],
                                                            kRealCin[l], kRealCout[l], kCin[l], kCout[l], lr, b1,
                                                            b2, eps, c1, c2, net->Bt[l], net->Bf[l]);
        CNN_CUDA(net, cudaGetLastError());
        k_adam_bias<<<1, 32, 0, net->st>>>(net->b[l], net->mb[l], net->vb[l], net->gB[l], kRealCout[l], lr, b1, b2,
                                          eps, c1, c2);
        CNN_CUDA(net, cudaGetLastError());
    }
    return LEM_OK;
}

}  // extern "C"

namespace lem {
int cnn_forward_on(lem_cnn *net, const float *x, int H4, int W4, float *y, cudaStream_t st) {
    cudaStream_t keep = net->st;
    net->st = st;
    const int rc = lem_cnn_forward(net, x, H4, W4, y);
    net->st = keep;
    return rc;
}
const char *cnn_error(const lem_cnn *net) { return lem_cnn_last_error(net); }
}  // namespace lem
