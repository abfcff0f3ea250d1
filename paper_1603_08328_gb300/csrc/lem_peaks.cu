// Microbenchmarks of the two on-chip roofs the data term is held against: FP32
// fused multiply-add throughput and shared-memory load bandwidth, measured on
// every SM of the current device (a measurement aid; the paper has no
// counterpart).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lem.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// kChains independent chains of `iters` FMAs per thread; the result is stored
// only when it matches a value it cannot take, so nothing is optimised away
__global__ void __launch_bounds__(256) k_peak_fma(float a0, float b, int iters, float *sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = a0 + (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], b, 1e-7f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.2345f) *sink = s;
}

// 16-byte shared-memory loads: thread t reads word (t + k * blockDim) of a
// 32 KiB array, so a warp's 32 loads fall in distinct bank groups
__global__ void __launch_bounds__(1024) k_peak_smem(int iters, float *sink) {
    constexpr int kWords = 2048;  // float4 words = 32 KiB
    __shared__ float4 buf[kWords];
    for (int i = threadIdx.x; i < kWords; i += blockDim.x) buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 v = buf[idx];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
            idx = (idx + blockDim.x) & (kWords - 1);
        }
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.2345f) *sink = acc.x;
}

// best (shortest) of `reps` timed launches of fn, in ms
template <typename F>
cudaError_t best_ms(F fn, cudaStream_t st, int reps, float *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = -1.f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = fn();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && r > 0 && (best < 0.f || t < best)) best = t;  // launch 0 warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms = best;
    return e;
}

}  // namespace

extern "C" int lem_measure_peaks(void *stream, double *fp32_tflops, double *smem_gbs) {
    if (!fp32_tflops || !smem_gbs) return LEM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LEM_ERR_CUDA;
    float *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return LEM_ERR_OOM;
    // FMA: 8 CTAs of 256 threads per SM (full occupancy), 16 * 8 FMAs per iteration
    const int fma_blocks = 8 * nsm, fma_iters = 4096;
    float ms_fma = 0.f, ms_smem = 0.f;
    cudaError_t e = best_ms(
        [&]() {
            k_peak_fma<<<fma_blocks, 256, 0, st>>>(1.0f, 0.999f, fma_iters, sink);
            return cudaGetLastError();
        },
        st, 6, &ms_fma);
    // shared memory: 2 CTAs of 1024 threads per SM, 8 loads of 16 bytes per iteration
    const int sm_blocks = 2 * nsm, sm_iters = 4096;
    if (e == cudaSuccess)
        e = best_ms(
            [&]() {
                k_peak_smem<<<sm_blocks, 1024, 0, st>>>(sm_iters, sink);
                return cudaGetLastError();
            },
            st, 6, &ms_smem);
    cudaFree(sink);
    if (e != cudaSuccess || ms_fma <= 0.f || ms_smem <= 0.f) return LEM_ERR_CUDA;
    const double flops = 2.0 * kChains * 16.0 * fma_iters * 256.0 * fma_blocks;
    const double bytes = 16.0 * 8.0 * sm_iters * 1024.0 * sm_blocks;
    *fp32_tflops = flops / (ms_fma * 1e-3) / 1e12;
    *smem_gbs = bytes / (ms_smem * 1e-3) / 1e9;
    return LEM_OK;
}
