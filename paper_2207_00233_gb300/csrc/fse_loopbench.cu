// Microbenchmark of the FSE iteration loop alone (Sec. 4: K selections and
// transform-domain residual updates of one block's 64x64 spectrum), with
// the selection step in one of three exact forms.  It times the loop body of
// the per-block kernels (the same device functions, fse_iter.cuh) with the
// same CTA shape, shared-memory table and register layout, at a chosen
// number of CTAs per SM, without the gather, projection and synthesis.  All
// forms select the same indices (ties to the smallest linear index); a
// checksum of the selected indices lets the caller verify that.
//
// Inputs are generated in the kernel: W = DFT64 of the separable positive
// weight a[m] a[n], a[m] = 0.7^|m - 23.5| (48 samples), which keeps the
// iteration's energy decreasing as in FSE; R_w starts as pseudo-random
// values.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/fse.h"
#include "fse_iter.cuh"

namespace {

using namespace fse;
using namespace fse::iter;

constexpr int kLbSlotOff = kW4Bytes;                  // 2 x 8 uint4: one-barrier slots
                                                      // (variant 3: the first two)
constexpr int kLbSmaxOff = kLbSlotOff + 2 * kWarps * 16;  // 8 words: warp maxima
constexpr int kLbCandOff = kLbSmaxOff + kWarps * 4;   // 8 float4: two-barrier candidates
constexpr int kLbAOff = kLbCandOff + kWarps * 16;     // 64 float2: 1-D DFT of a
constexpr int kLbListOff = kLbAOff + kDft * 8;        // dc list [K] float2, u list [K] u16
inline int lb_smem_bytes(int iters) { return kLbListOff + iters * 8 + ((iters * 2 + 15) / 16) * 16; }

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ void build_w4(unsigned char *smem) {
    float2 *A = reinterpret_cast<float2 *>(smem + kLbAOff);
    const int tid = threadIdx.x;
    if (tid < kDft) {
        float re = 0.f, im = 0.f;
        for (int m = 0; m < kArea; ++m) {
            const float a = powf(0.7f, fabsf((float)m - 23.5f));
            float s, c;
            sincospif((float)((tid * m) & (kDft - 1)) / 32.f, &s, &c);
            re = fmaf(a, c, re);
            im = fmaf(-a, s, im);
        }
        A[tid] = make_float2(re, im);
    }
    __syncthreads();
    float4 *w4 = reinterpret_cast<float4 *>(smem);
    for (int e = tid; e < kW4Rows * kDft; e += kThreads) {
        const int row = (e / kDft) & (kDft - 1), j = e % kDft;
        const float2 a = A[row], b = A[j], b2 = A[j ^ 32];
        const float wr = a.x * b.x - a.y * b.y, wi = a.x * b.y + a.y * b.x;
        const float wr2 = a.x * b2.x - a.y * b2.y, wi2 = a.x * b2.y + a.y * b2.x;
        w4[e] = make_float4(wr, wr2, wi, wi2);
    }
    __syncthreads();
}

template <int V>
__global__ void __launch_bounds__(kThreads, 3)
k_loop(int iters, int blocks, float gamma, uint32_t *sums) {
    extern __shared__ __align__(128) unsigned char smem[];
    build_w4(smem);
    const int tid = threadIdx.x;
    const float W0 = reinterpret_cast<const float4 *>(smem)[0].x;
    const float gw = gamma / W0;
    const uint32_t w4addr = smem_addr(smem);
    uint4 *slots = reinterpret_cast<uint4 *>(smem + kLbSlotOff);
    uint32_t *smax = reinterpret_cast<uint32_t *>(smem + kLbSmaxOff);
    float4 *cand = reinterpret_cast<float4 *>(smem + kLbCandOff);
    float2 *dcl = reinterpret_cast<float2 *>(smem + kLbListOff);
    uint16_t *ul = reinterpret_cast<uint16_t *>(smem + kLbListOff + iters * 8);
    uint32_t sum = 0;
    for (int b = 0; b < blocks; ++b) {
        u64 rre[8], rim[8];
        const uint32_t seed = (blockIdx.x * blocks + b) * kThreads + tid;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint32_t h = hash32(seed * 16 + 2 * r), g = hash32(seed * 16 + 2 * r + 1);
            rre[r] = pack2((h & 0xffff) * (1.f / 655.36f), (h >> 16) * (1.f / 655.36f));
            rim[r] = pack2((g & 0xffff) * (1.f / 655.36f) - 50.f, (g >> 16) * (1.f / 655.36f) - 50.f);
        }
        if (V == 5 || V == 6) {
            // Calibration forms, not FSE: the index sequence is fixed
            // (u = hash of the iteration), so no selection is made; variant 6
            // adds the warp reduction and one block barrier per iteration.
            u64 ndcr2 = 0ull, dci2 = 0ull, ndci2 = 0ull;
            uint32_t wbase = w4_base(w4addr, 0, 0);
            uint32_t acc = 0;
            for (int it = 0; it < iters; ++it) {
                const float tmx = update_and_max(wbase, ndcr2, dci2, ndci2, rre, rim);
                uint32_t v = __float_as_uint(tmx);
                if (V == 6) {
                    v = __reduce_max_sync(0xffffffffu, v);
                    if ((tid & 31) == 0) smax[tid >> 5] = v;
                    __syncthreads();
                    v = __reduce_max_sync(0xffffffffu, smax[tid & 7]);
                }
                acc += v;
                // (v >> 31 is 0: energies are not negative; it makes the next
                // iteration depend on this one's update, as a selection does)
                const uint32_t u = ((it * 2654435761u + b * 40503u) >> 20 ^ (v >> 31)) & 4095u;
                const float dcr = 1e-3f * (float)(u & 15), dci = -1e-3f * (float)(u >> 8);
                ndcr2 = pack2(-dcr, -dcr);
                dci2 = pack2(dci, dci);
                ndci2 = pack2(-dci, -dci);
                wbase = w4_base(w4addr, (int)(u >> 6), (int)(u & 63));
                if (V == 6) __syncthreads();  // smax is rewritten next iteration
            }
            if (tid == 0) sum += acc;
            continue;
        }
        if (V == 3 || V == 4) {
            const uint32_t w8k = (uint32_t)(8 * (tid >> 5)) << 10, l16 = (uint32_t)(tid & 31) << 4;
            Step st{0ull, 0ull, 0ull, 0u, 0u};  // first pass: dc = 0
            for (int it = 0; it < iters; ++it) {
                const uint32_t wb = w4_addr_of(w4addr, w8k, l16, st);
                const float tmx = update_and_max(wb, st.ndcr2, st.dci2, st.ndci2, rre, rim);
                select_named_warp<V == 4>(tmx, rre, rim, gw, it, smax, slots, dcl, ul, st);
                if (tid == 0) sum = sum * 1000003u + ul[it];
            }
            __syncthreads();
            if (tid == 0) sum += ul[iters - 1];
            __syncthreads();
            continue;
        }
        u64 ndcr2 = 0ull, dci2 = 0ull, ndci2 = 0ull;
        uint32_t wbase = w4_base(w4addr, 0, 0);
        for (int it = 0; it < iters; ++it) {
            uint32_t u;
            float ure, uim;
            if (V == 0) {
                const float tmx = update_and_max(wbase, ndcr2, dci2, ndci2, rre, rim);
                select_two_barriers(tmx, rre, rim, smax, cand, u, ure, uim);
            } else if (V == 1) {
                uint32_t wm;
                int rs;
                update_rowmax(wbase, ndcr2, dci2, ndci2, rre, rim, wm, rs);
                uint4 *sl = slots + (it & 1) * kWarps;
                publish_row_candidate(wm, rs, rre, rim, sl);
                __syncthreads();
                pick_candidate(sl, u, ure, uim);
            } else {
                const float tmx = update_and_max(wbase, ndcr2, dci2, ndci2, rre, rim);
                uint4 *sl = slots + (it & 1) * kWarps;
                publish_searched_candidate(tmx, rre, rim, sl);
                __syncthreads();
                pick_candidate(sl, u, ure, uim);
            }
            const float dcr = ure * gw, dci = uim * gw;
            if (tid == 0) {
                dcl[it] = make_float2(dcr, dci);
                ul[it] = (uint16_t)u;
                sum = sum * 1000003u + u;
            }
            ndcr2 = pack2(-dcr, -dcr);
            dci2 = pack2(dci, dci);
            ndci2 = pack2(-dci, -dci);
            wbase = w4_base(w4addr, (int)(u >> 6), (int)(u & 63));
        }
        __syncthreads();
        if (tid == 0) sum += ul[iters - 1];
        __syncthreads();
    }
    if (tid == 0) sums[blockIdx.x] = sum;
}

template <int V>
cudaError_t prepare(int smem, int ctas, int *fit) {
    cudaError_t e = cudaFuncSetAttribute(k_loop<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(fit, k_loop<V>, kThreads, smem);
}

}  // namespace

extern "C" int fse_loop_microbench(int device, int variant, int ctas_per_sm, int iters,
                                   int blocks_per_cta, double *ns_per_block_iter,
                                   uint32_t *checksum) {
    if (!ns_per_block_iter || !checksum || variant < 0 || variant > 6 || ctas_per_sm < 1 ||
        iters < 1 || iters > FSE_MAX_ITERS || blocks_per_cta < 1 || blocks_per_cta > 4096)
        return FSE_EINVAL;
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
    const int smem = lb_smem_bytes(iters);
    int fit = 0;
    cudaError_t e = variant == 0   ? prepare<0>(smem, ctas_per_sm, &fit)
                    : variant == 1 ? prepare<1>(smem, ctas_per_sm, &fit)
                    : variant == 2 ? prepare<2>(smem, ctas_per_sm, &fit)
                    : variant == 3 ? prepare<3>(smem, ctas_per_sm, &fit)
                    : variant == 4 ? prepare<4>(smem, ctas_per_sm, &fit)
                    : variant == 5 ? prepare<5>(smem, ctas_per_sm, &fit)
                                   : prepare<6>(smem, ctas_per_sm, &fit);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FSE_ECUDA;
    }
    if (ctas_per_sm > fit) return FSE_EINVAL;  // would not be resident at once
    const int grid = sms * ctas_per_sm;
    uint32_t *sums = nullptr;
    if (cudaMalloc(&sums, sizeof(uint32_t) * grid) != cudaSuccess) {
        cudaGetLastError();
        return FSE_ENOMEM;
    }
    auto launch = [&] {
        if (variant == 0)
            k_loop<0><<<grid, kThreads, smem>>>(iters, blocks_per_cta, 0.5f, sums);
        else if (variant == 1)
            k_loop<1><<<grid, kThreads, smem>>>(iters, blocks_per_cta, 0.5f, sums);
        else if (variant == 2)
            k_loop<2><<<grid, kThreads, smem>>>(iters, blocks_per_cta, 0.5f, sums);
        else if (variant == 3)
            k_loop<3><<<grid, kThreads, smem>>>(iters, blocks_per_cta, 0.5f, sums);
        else if (variant == 4)
            k_loop<4><<<grid, kThreads, smem>>>(iters, blocks_per_cta, 0.5f, sums);
        else if (variant == 5)
            k_loop<5><<<grid, kThreads, smem>>>(iters, blocks_per_cta, 0.5f, sums);
        else
            k_loop<6><<<grid, kThreads, smem>>>(iters, blocks_per_cta, 0.5f, sums);
    };
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = FSE_OK;
    float ms = 0.f;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        rc = FSE_ECUDA;
    } else {
        launch();
        cudaEventRecord(a);
        launch();
        cudaEventRecord(b);
        if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
            rc = FSE_ECUDA;
    }
    std::vector<uint32_t> h(grid);
    if (rc == FSE_OK &&
        cudaMemcpy(h.data(), sums, sizeof(uint32_t) * grid, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = FSE_ECUDA;
    if (rc == FSE_OK) {
        uint32_t c = 0;
        for (int i = 0; i < grid; ++i) c = c * 31u + h[i];
        *checksum = c;
        *ns_per_block_iter =
            (double)ms * 1e6 * sms / ((double)grid * blocks_per_cta * iters);
    }
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(sums);
    return rc;
}
