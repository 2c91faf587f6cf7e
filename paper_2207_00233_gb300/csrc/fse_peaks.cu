// Measured ceilings of the units the FSE iteration loop runs on: shared-memory
// load bandwidth (16-byte loads, conflict-free, every SM) and FP32 fused
// multiply-add throughput (packed f32x2, every SM).  The roofline of the hot
// kernel is reported against these; the device's nominal figures are not
// published per unit for this part.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/fse.h"

namespace {

constexpr int kLdsThreads = 512;
constexpr int kLdsWords = 4096;  // uint4 entries: 64 KB of shared memory

// Each thread streams 16-byte loads over a 64 KB table: lane l of a warp reads
// entry (base + l), so a warp's request covers 512 contiguous bytes (four
// 128-byte wavefronts, no bank conflicts).  The XOR of everything read is
// stored only when it matches an impossible pattern, so the loads stay live.
__global__ void __launch_bounds__(kLdsThreads) k_lds_stream(int iters, uint32_t *sink) {
    extern __shared__ uint4 tab[];
    for (int i = threadIdx.x; i < kLdsWords; i += blockDim.x)
        tab[i] = make_uint4(i * 2654435761u, i ^ 0x9e3779b9u, i * 40503u, ~i);
    __syncthreads();
    uint32_t acc = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int base = warp * 256;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint4 v = tab[(base + 32 * k + lane) & (kLdsWords - 1)];
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
        base = (base + 256 + it) & (kLdsWords - 1);
    }
    if (acc == 0x7f3a5c1du) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// Eight independent packed f32x2 FMA chains per thread.
__global__ void __launch_bounds__(256) k_ffma2(int iters, float *sink) {
    unsigned long long a[8];
    const float s = 1.0f + 1e-7f * threadIdx.x;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float x = 0.5f + 0.01f * k, y = 0.25f + 0.02f * k;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(x), "f"(y));
    }
    unsigned long long m, c;
    asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(s));
    asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(1e-6f));
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(m), "l"(c));
        }
    }
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[k]));
        t += x + y;
    }
    if (t == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// Runs `launch` twice (the first as warm-up) and returns the second's
// milliseconds, or a negative value on error.
template <class F>
float time_launch(F launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaEventDestroy(a);
        return -1.f;
    }
    float ms = -1.f;
    launch();
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    if (cudaEventSynchronize(b) == cudaSuccess && cudaGetLastError() == cudaSuccess)
        cudaEventElapsedTime(&ms, a, b);
    else
        cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

extern "C" int fse_measure_peaks(int device, double *smem_gbs, double *fp32_tflops) {
    if (!smem_gbs || !fp32_tflops) return FSE_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    if (device < 0 || device >= ndev) return FSE_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    const int lds_smem = kLdsWords * (int)sizeof(uint4);
    if (cudaFuncSetAttribute(k_lds_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             lds_smem) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    int lds_per_sm = 0, fma_per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lds_per_sm, k_lds_stream, kLdsThreads,
                                                      lds_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fma_per_sm, k_ffma2, 256, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    const int lds_grid = sms * (lds_per_sm > 0 ? lds_per_sm : 1);
    const int fma_grid = sms * (fma_per_sm > 0 ? fma_per_sm : 1);
    void *sink = nullptr;
    const size_t sink_bytes = sizeof(float) * (size_t)std::max(lds_grid * kLdsThreads,
                                                                fma_grid * 256);
    if (cudaMalloc(&sink, sink_bytes) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ENOMEM;
    }
    const int lds_iters = 4096, fma_iters = 32;
    const float lds_ms = time_launch([&] {
        k_lds_stream<<<lds_grid, kLdsThreads, lds_smem>>>(lds_iters,
                                                          static_cast<uint32_t *>(sink));
    });
    const float fma_ms = time_launch([&] {
        k_ffma2<<<fma_grid, 256>>>(fma_iters, static_cast<float *>(sink));
    });
    cudaFree(sink);
    if (lds_ms <= 0.f || fma_ms <= 0.f) return FSE_ECUDA;
    const double lds_bytes = (double)lds_grid * kLdsThreads * lds_iters * 8 * 16;
    const double fma_flop = (double)fma_grid * 256 * fma_iters * 16 * 8 * 2 * 2;
    *smem_gbs = lds_bytes / (lds_ms * 1e-3) / 1e9;
    *fp32_tflops = fma_flop / (fma_ms * 1e-3) / 1e12;
    return FSE_OK;
}
