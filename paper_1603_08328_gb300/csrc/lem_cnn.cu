// Plane-proposal network: 6 layers of 3x3 convolutions (32 channels, ReLU
// between layers) on (left RGB, right RGB, disparity) at quarter resolution,
// predicting (d, a, b) per quarter-resolution pixel; bilinear upsampling turns
// the prediction into a full-resolution map of plane labels that the
// expansion kernel can draw candidates from.
//
// Convolutions are implicit GEMMs on the tensor cores (BF16 operands, FP32
// accumulation):
//   forward      Y[p][o]   = sum_k Xpatch[p][k] W[k][o]        (M = 128 pixels, N = Cout, K = 9 Cin)
//                on tcgen05.mma with the accumulator in tensor memory
//   input grad   dX        = the same kernel with flipped, transposed weights
//   weight grad  dW^T[k][o] = sum_p Xpatch[p][k] dZ[p][o]     (M = 9 Cin, N = Cout, K = pixels)
//                on tcgen05.mma: each CTA accumulates its pixel range in tensor
//                memory and writes a partial sum; a second kernel adds the
//                partials in a fixed order, so gradients are bit-reproducible
// Activations are BF16, NHWC, channels padded to a multiple of 16; the weights
// have an FP32 master copy updated by Adam.
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

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t ld_u32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

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

// Y = conv3x3(X) (+ bias) for 128 pixels per CTA as one 128 x COUT x 9CIN GEMM
// on the tensor cores: the pixels' 3x3 patches (A, 128 x K) and the weights
// (B, COUT x K, both K-major) are staged in shared memory, one thread issues
// K/16 tcgen05.mma into a TMEM accumulator, and each warp reads its 32 rows
// back for the epilogue.
// B images of H x W pixels are stacked row after row; a patch never reaches
// across an image's border (zero padding as for a single image).
//   X  : B*H*W*CIN bf16;  Bt : COUT x (9 CIN) bf16 (row o holds W[k][o]);
//   Z  : optional fp32 pre-activation B*H*W*COUT;  Y : optional bf16 output (ReLU if relu)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_conv(const bf16 *X, int H, int W, int B, const bf16 *Bt,
                                                       const float *bias, float *Z, bf16 *Y, int relu) {
    constexpr int K = 9 * CIN, KC = K / 8, CH = CIN / 8;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *As = sm_raw;                          // 128 x K, core-matrix layout
    unsigned char *Bs = sm_raw + (size_t)kTileP * K * 2; // COUT x K, core-matrix layout
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = H * W * B, p0 = blockIdx.x * kTileP;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // weights: row o, k chunk c -> core matrix (o/8, c), row o%8
    for (int q = tid; q < COUT * KC; q += kConvThreads) {
        const int o = q / KC, c = q - o * KC;
        *reinterpret_cast<uint4 *>(Bs + ((o >> 3) * KC + c) * 128 + (o & 7) * 16) =
            *reinterpret_cast<const uint4 *>(Bt + (size_t)o * K + c * 8);
    }
    // patches: one thread per pixel row r, k chunk c = tap * CH + c8
    {
        const int r = tid, p = p0 + r;
        unsigned char *row = As + (size_t)(r >> 3) * KC * 128 + (r & 7) * 16;
        const int u = p % W, y = p / W, v = y % H;  // row of the stacked images, row within the image
        for (int c = 0; c < KC; ++c) {
            const int tap = c / CH, c8 = c - tap * CH;
            const int uu = u + tap % 3 - 1, dv = tap / 3 - 1;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (p < n && uu >= 0 && uu < W && v + dv >= 0 && v + dv < H)
                val = *reinterpret_cast<const uint4 *>(X + ((size_t)(y + dv) * W + uu) * CIN + c8 * 8);
            *reinterpret_cast<uint4 *>(row + c * 128) = val;
        }
    }
    // generic-proxy stores -> visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = tmem_base;
    if (tid == 0) {
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
        constexpr uint32_t idesc = idesc_bf16(kTileP, COUT);
#pragma unroll 1
        for (int kk = 0; kk < K / 16; ++kk) {
            // K step kk covers core-matrix columns 2kk, 2kk+1
            const uint64_t ad = smem_desc(a0 + kk * 256, 128, KC * 128);
            const uint64_t bd = smem_desc(b0 + kk * 256, 128, KC * 128);
            mma_tc(tbase, ad, bd, idesc, kk > 0 ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&mbar))
                     : "memory");
    }
    const bool ok = mbar_wait0(smem_u32(&mbar), kMmaWaitLimit);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        float acc[COUT];
        tmem_load_row<COUT>(tbase + ((uint32_t)(warp * 32) << 16), acc);
        const int p = p0 + warp * 32 + lane;
        if (p < n) {
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] += bias ? bias[o] : 0.f;
            if (Z) {
                float4 *z4 = reinterpret_cast<float4 *>(Z + (size_t)p * COUT);
#pragma unroll
                for (int o = 0; o < COUT; o += 4) z4[o / 4] = make_float4(acc[o], acc[o + 1], acc[o + 2], acc[o + 3]);
            }
            if (Y) {
                uint4 *y4 = reinterpret_cast<uint4 *>(Y + (size_t)p * COUT);
#pragma unroll
                for (int o = 0; o < COUT; o += 8) {
                    __nv_bfloat162 h[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float x0 = relu ? fmaxf(acc[o + 2 * j], 0.f) : acc[o + 2 * j];
                        const float x1 = relu ? fmaxf(acc[o + 2 * j + 1], 0.f) : acc[o + 2 * j + 1];
                        h[j] = __floats2bfloat162_rn(x0, x1);
                    }
                    y4[o / 8] = *reinterpret_cast<uint4 *>(h);
                }
            }
        }
    } else if (tid == 0) {
        atomicAdd(&g_mma_timeouts, 1u);
        // give the MMAs in flight one more bounded chance before TMEM is freed
        mbar_wait0(smem_u32(&mbar), kMmaWaitLimit);
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
//   X  : B*H*W*CIN bf16 (B stacked images, as in k_conv);  dZ : B*H*W*COUT bf16
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads) k_wgrad_tc(const bf16 *X, const bf16 *dZ, int H, int W, int B,
                                                           int tiles_per_cta, float *part, float *partb) {
    constexpr int K = 9 * CIN, MT = (K + 127) / 128, MP = MT * 128, PC = kTileP / 8, CH = CIN / 8;
    constexpr int TC = MT * COUT <= 32 ? 32 : (MT * COUT <= 64 ? 64 : (MT * COUT <= 128 ? 128 : 256));
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *As = sm_raw;                             // MP x 128 pixels
    unsigned char *Bs = sm_raw + (size_t)MP * kTileP * 2;   // COUT x 128 pixels
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float s_db[COUT];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = H * W * B;
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
            const int u = p % W, y = p / W, v = y % H;  // as in k_conv
            for (int c = 0; c < 9 * CH; ++c) {
                const int tap = c / CH, c8 = c - tap * CH;
                const int uu = u + tap % 3 - 1, dv = tap / 3 - 1;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (p < n && uu >= 0 && uu < W && v + dv >= 0 && v + dv < H)
                    val = *reinterpret_cast<const uint4 *>(X + ((size_t)(y + dv) * W + uu) * CIN + c8 * 8);
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
                if (p < n) val = *reinterpret_cast<const uint4 *>(dZ + (size_t)p * COUT + c8 * 8);
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

// dZprev = dX * (Zprev > 0) as bf16 (ReLU backward); channels padded
__global__ void k_relu_back(const float *dX, const float *Zprev, int count, bf16 *dZ) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    dZ[i] = __float2bfloat16_rn(Zprev[i] > 0.f ? dX[i] : 0.f);
}

// L1 loss on (d, a, b): out is H*W*16 fp32 (channels 0..2 used), target H*W*3;
// writes d loss / d out (bf16, padded channels zero) and accumulates the loss
__global__ void k_l1_loss(const float *out, const float *target, int n, float s0, float s1, float s2, float inv_n,
                          bf16 *dout, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (p < n) {
        const float sc[3] = {s0, s1, s2};
        for (int c = 0; c < 16; ++c) {
            float gval = 0.f;
            if (c < 3) {
                const float diff = out[(size_t)p * 16 + c] - target[(size_t)p * 3 + c];
                l += sc[c] * fabsf(diff);
                gval = (diff > 0.f ? sc[c] : (diff < 0.f ? -sc[c] : 0.f)) * inv_n;
            }
            dout[(size_t)p * 16 + c] = __float2bfloat16_rn(gval);
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l * inv_n);
}

// Adam on the fp32 master weights of one layer (real channels only), then the
// bf16 copies: forward Bt[o][k] and input-gradient Bf[c][k'] (flipped taps,
// roles of channels swapped).
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
    Bt[(size_t)o * 9 * CIN + tap * CIN + c] = __float2bfloat16_rn(wn);
    if (Bf) Bf[(size_t)c * 9 * COUT + (8 - tap) * COUT + o] = __float2bfloat16_rn(wn);
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
    Bt[(size_t)o * 9 * CIN + tap * CIN + c] = __float2bfloat16_rn(w[idx]);
    if (Bf) Bf[(size_t)c * 9 * COUT + (8 - tap) * COUT + o] = __float2bfloat16_rn(w[idx]);
}

// quarter-resolution input: x (fp32, H4*W4*7: R,G,B of left, R,G,B of right /255,
// disparity / dmax) -> bf16 padded to 16 channels
__global__ void k_pack_input(const float *x, int n, bf16 *X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * 16) return;
    const int p = i / 16, c = i % 16;
    X[i] = __float2bfloat16_rn(c < 7 ? x[(size_t)p * 7 + c] : 0.f);
}

// network output (pre-activation of the last layer, 16 padded channels) -> y (3 channels)
__global__ void k_take3(const float *z, int n, float *y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * 3) return;
    y[i] = z[(size_t)(i / 3) * 16 + i % 3];
}

template <int CIN, int COUT>
size_t conv_smem() {
    return (size_t)2 * 9 * CIN * (kTileP + COUT);
}
constexpr int kWgParts = 148;  // most CTAs (partial sums) of one weight-gradient launch

template <int CIN, int COUT>
size_t wgrad_smem() {
    return (size_t)2 * kTileP * ((9 * CIN + 127) / 128 * 128 + COUT);
}

template <int CIN, int COUT>
cudaError_t conv(const bf16 *X, int H, int W, int B, const bf16 *Bt, const float *bias, float *Z, bf16 *Y,
                 int relu, cudaStream_t st) {
    const size_t sm = conv_smem<CIN, COUT>();
    cudaError_t e = cudaFuncSetAttribute(k_conv<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nb = (H * W * B + kTileP - 1) / kTileP;
    k_conv<CIN, COUT><<<nb, kConvThreads, sm, st>>>(X, H, W, B, Bt, bias, Z, Y, relu);
    return cudaGetLastError();
}

// part: kWgParts * COUT * 9CIN floats, partb: kWgParts * COUT floats (scratch)
template <int CIN, int COUT>
cudaError_t wgrad(const bf16 *X, const bf16 *dZ, int H, int W, int B, float *dW, float *dB, float *part,
                  float *partb, cudaStream_t st) {
    const size_t sm = wgrad_smem<CIN, COUT>();
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int tiles = (H * W * B + kTileP - 1) / kTileP;
    const int per = (tiles + kWgParts - 1) / kWgParts;
    const int G = (tiles + per - 1) / per;
    k_wgrad_tc<CIN, COUT><<<G, kConvThreads, sm, st>>>(X, dZ, H, W, B, per, part, partb);
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
    // activations of up to cap pixels (all images of a training step, stacked)
    size_t cap = 0;
    bf16 *act[kLayers + 1] = {};                  // layer inputs (bf16), act[0] = packed input
    float *pre[kLayers] = {};                     // pre-activations (fp32)
    bf16 *dz = nullptr;                           // d loss / d pre-activation (bf16, 32 ch)
    float *dx = nullptr;                          // d loss / d layer input (fp32, 32 ch)
    float *loss = nullptr;
    float *xin = nullptr, *tgt = nullptr;         // staging of an input / target
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

int ensure_capacity(lem_cnn *net, size_t npix) {
    if (npix <= net->cap) return LEM_OK;
    // pointers are cleared as they are freed, so a failed allocation below
    // leaves nothing dangling for a later call or lem_cnn_destroy
    auto drop = [](auto *&p) {
        cudaFree(p);
        p = nullptr;
    };
    net->cap = 0;
    for (int l = 0; l <= kLayers; ++l) drop(net->act[l]);
    for (int l = 0; l < kLayers; ++l) drop(net->pre[l]);
    drop(net->dz);
    drop(net->dx);
    drop(net->xin);
    drop(net->tgt);
    for (int l = 0; l <= kLayers; ++l) {
        const int c = l == 0 ? kCin[0] : kCout[l - 1];
        CNN_CUDA(net, cudaMalloc(&net->act[l], sizeof(bf16) * npix * c));
    }
    for (int l = 0; l < kLayers; ++l) CNN_CUDA(net, cudaMalloc(&net->pre[l], sizeof(float) * npix * kCout[l]));
    CNN_CUDA(net, cudaMalloc(&net->dz, sizeof(bf16) * npix * 32));
    CNN_CUDA(net, cudaMalloc(&net->dx, sizeof(float) * npix * 32));
    CNN_CUDA(net, cudaMalloc(&net->xin, sizeof(float) * npix * 7));
    CNN_CUDA(net, cudaMalloc(&net->tgt, sizeof(float) * npix * 3));
    net->cap = npix;
    return LEM_OK;
}

cudaError_t forward(lem_cnn *net, int H4, int W4, int B) {
    cudaStream_t st = net->st;
    cudaError_t e = conv<16, 32>(net->act[0], H4, W4, B, net->Bt[0], net->b[0], net->pre[0], net->act[1], 1, st);
    for (int l = 1; l < 5 && e == cudaSuccess; ++l)
        e = conv<32, 32>(net->act[l], H4, W4, B, net->Bt[l], net->b[l], net->pre[l], net->act[l + 1], 1, st);
    if (e == cudaSuccess) e = conv<32, 16>(net->act[5], H4, W4, B, net->Bt[5], net->b[5], net->pre[5], nullptr, 0, st);
    return e;
}

// backward of B stacked images from d loss / d output (in net->dz, 16
// channels); accumulates into gW / gB
cudaError_t backward(lem_cnn *net, int H4, int W4, int B) {
    cudaStream_t st = net->st;
    const int n = H4 * W4 * B;
    cudaError_t e = cudaSuccess;
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
        // weight gradient of layer l: input act[l], output gradient dz
        if (l == 5)
            e = wgrad<32, 16>(net->act[5], net->dz, H4, W4, B, net->gW[5], net->gB[5], net->wpart, net->wpartb, st);
        else if (l == 0)
            e = wgrad<16, 32>(net->act[0], net->dz, H4, W4, B, net->gW[0], net->gB[0], net->wpart, net->wpartb, st);
        else
            e = wgrad<32, 32>(net->act[l], net->dz, H4, W4, B, net->gW[l], net->gB[l], net->wpart, net->wpartb, st);
        if (e != cudaSuccess || l == 0) break;
        // input gradient: conv of dz with the flipped, transposed weights
        if (l == 5) e = conv<16, 32>(net->dz, H4, W4, B, net->Bf[5], nullptr, net->dx, nullptr, 0, st);
        else e = conv<32, 32>(net->dz, H4, W4, B, net->Bf[l], nullptr, net->dx, nullptr, 0, st);
        if (e != cudaSuccess) break;
        // ReLU of layer l-1
        const int cnt = n * kCout[l - 1];
        k_relu_back<<<(cnt + 255) / 256, 256, 0, st>>>(net->dx, net->pre[l - 1], cnt, net->dz);
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
    for (int l = 0; l <= kLayers; ++l) cudaFree(net->act[l]);
    cudaFree(net->dz);
    cudaFree(net->dx);
    cudaFree(net->loss);
    cudaFree(net->wpart);
    cudaFree(net->wpartb);
    cudaFree(net->xin);
    cudaFree(net->tgt);
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
    const size_t n = (size_t)H4 * W4;
    int rc = ensure_capacity(net, n);
    if (rc != LEM_OK) return rc;
    k_pack_input<<<(int)((n * 16 + 255) / 256), 256, 0, net->st>>>(x, (int)n, net->act[0]);
    CNN_CUDA(net, cudaGetLastError());
    CNN_CUDA(net, forward(net, H4, W4, 1));
    k_take3<<<(int)((n * 3 + 255) / 256), 256, 0, net->st>>>(net->pre[5], (int)n, out);
    CNN_CUDA(net, cudaGetLastError());
    return LEM_OK;
}

int lem_cnn_gradients(lem_cnn *net, const float *x, const float *target, int n_images, int H4, int W4,
                      const float *scale, float *loss, float *grads) {
    if (!net || !x || !target || n_images < 1 || H4 < 1 || W4 < 1 || !scale) return LEM_ERR_ARG;
    // all images go through each layer in one launch: the batch is stacked as
    // one (n_images * H4) x W4 grid whose patches stop at each image's border
    const size_t n = (size_t)H4 * W4 * n_images;
    if (n * 32 > (size_t)INT32_MAX) return LEM_ERR_ARG;
    int rc = ensure_capacity(net, n);
    if (rc != LEM_OK) return rc;
    for (int l = 0; l < kLayers; ++l) {
        CNN_CUDA(net, cudaMemsetAsync(net->gW[l], 0, sizeof(float) * kCout[l] * 9 * kCin[l], net->st));
        CNN_CUDA(net, cudaMemsetAsync(net->gB[l], 0, sizeof(float) * kCout[l], net->st));
    }
    CNN_CUDA(net, cudaMemsetAsync(net->loss, 0, sizeof(float), net->st));
    const float inv_n = 1.f / (float)n;
    k_pack_input<<<(int)((n * 16 + 255) / 256), 256, 0, net->st>>>(x, (int)n, net->act[0]);
    CNN_CUDA(net, cudaGetLastError());
    CNN_CUDA(net, forward(net, H4, W4, n_images));
    k_l1_loss<<<(int)((n + 255) / 256), 256, 0, net->st>>>(net->pre[5], target, (int)n, scale[0], scale[1], scale[2],
                                                         inv_n, net->dz, net->loss);
    CNN_CUDA(net, cudaGetLastError());
    CNN_CUDA(net, backward(net, H4, W4, n_images));
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
