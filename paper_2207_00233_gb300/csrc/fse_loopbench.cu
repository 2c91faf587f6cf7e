// Microbenchmark of the FSE iteration loop alone (Sec. 4: K selections and
// transform-domain residual updates of one block's 64x64 spectrum), with
// the selection step in one of several exact forms.  It times the loop body of
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

// Starting spectrum of block `seed`: entry (k_m, k_n) from a hash of its
// linear index, so that every thread layout starts from the same values.
// Thread (w, l) holds rows k_m = R w + r, columns l and l + 32.
template <int R>
__device__ __forceinline__ void init_spectrum(uint32_t seed, u64 (&rre)[R], u64 (&rim)[R]) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t k = seed * 4096u + (uint32_t)((R * w + r) * kDft + l);
        const uint32_t h0 = hash32(k), h1 = hash32(k + 32u);
        rre[r] = pack2((h0 & 0xffff) * (1.f / 655.36f), (h1 & 0xffff) * (1.f / 655.36f));
        rim[r] = pack2((h0 >> 16) * (1.f / 655.36f) - 50.f, (h1 >> 16) * (1.f / 655.36f) - 50.f);
    }
}

// The 1-D DFT of the separable weight a[m] = 0.7^|m - 23.5| (48 samples).
__device__ void build_a(float2 *A) {
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
}

__device__ void build_w4(unsigned char *smem) {
    float2 *A = reinterpret_cast<float2 *>(smem + kLbAOff);
    const int tid = threadIdx.x;
    build_a(A);
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
        init_spectrum<8>(blockIdx.x * blocks + b, rre, rim);
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
        if (V == 8) {  // the two maximum words start at zero
            if (tid < 2) smax[tid] = 0u;
            __syncthreads();
        }
        u64 ndcr2 = 0ull, dci2 = 0ull, ndci2 = 0ull;
        uint32_t wbase = w4_base(w4addr, 0, 0);
        for (int it = 0; it < iters; ++it) {
            uint32_t u;
            float ure, uim;
            if (V == 0) {
                const float tmx = update_and_max(wbase, ndcr2, dci2, ndci2, rre, rim);
                select_two_barriers(tmx, rre, rim, smax, cand, u, ure, uim);
            } else if (V == 7 || V == 8) {
                const float tmx = update_and_max(wbase, ndcr2, dci2, ndci2, rre, rim);
                select_two_barriers_v2<V == 8>(tmx, rre, rim, smax, cand, it, u, ure, uim);
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

// ---- planar W: variants 9 (256 threads, 8 rows per warp, 4 CTAs per SM)
// and 10 (128 threads, 16 rows per warp, 5 CTAs per SM) ----------------------
//
// W is kept once, as a plane of real and a plane of imaginary parts
// ([rows][64] floats each; rows 0..R-2 repeated after row 63), 36-40 KB
// instead of the 72.7 KB of the duplicated W4 layout, so more CTAs fit an
// SM.  A thread loads Re W and Im W at its two columns with four 4-byte
// loads per row (one wavefront each, as one 16-byte W4 load takes four) and
// the update is the same arithmetic as in the W4 forms, so every form
// selects the same indices.
template <int kT>
struct Planar {
    static constexpr int kNW = kT / 32;               // warps
    static constexpr int kR = kDft / kNW;             // rows per warp
    static constexpr int kRows = kDft + kR - 1;       // rows with the repeats
    static constexpr int kPlane = kRows * kDft * 4;   // bytes per plane
    static constexpr int kSmaxOff = 2 * kPlane;       // kNW words
    static constexpr int kCandOff = kSmaxOff + 32;    // kNW float4
    static constexpr int kAOff = kCandOff + 8 * 16;   // 64 float2
    static constexpr int kListOff = kAOff + kDft * 8;
    static int smem_bytes(int iters) { return kListOff + iters * 8 + ((iters * 2 + 15) / 16) * 16; }
};

template <int R, int NW>
__device__ __forceinline__ void select_planar(float tmx, const u64 (&rre)[R], const u64 (&rim)[R],
                                              uint32_t *smax, float4 *cand, uint32_t &u,
                                              float &ure, float &uim) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(tmx));
    if (l == 0) smax[w] = wmx;
    __syncthreads();
    const uint32_t estar = __reduce_max_sync(0xffffffffu, smax[l & (NW - 1)]);
    if (__any_sync(0xffffffffu, __float_as_uint(tmx) == estar)) {
        uint32_t kk = 0xffffffffu;
        float cre = 0.f, cim = 0.f;
        if (__float_as_uint(tmx) == estar) {
#pragma unroll
            for (int r = R - 1; r >= 0; --r) {
                const float2 e = unpack2(energy2(rre[r], rim[r]));
                const float2 re = unpack2(rre[r]), im = unpack2(rim[r]);
                if (__float_as_uint(e.y) == estar) {
                    kk = (uint32_t)((R * w + r) * kDft + l + 32);
                    cre = re.y;
                    cim = im.y;
                }
                if (__float_as_uint(e.x) == estar) {
                    kk = (uint32_t)((R * w + r) * kDft + l);
                    cre = re.x;
                    cim = im.x;
                }
            }
        }
        const uint32_t wk = __reduce_min_sync(0xffffffffu, kk);
        if (kk == wk) cand[w] = make_float4(__uint_as_float(wk), cre, cim, 0.f);
    } else if (l == 0) {
        cand[w].x = __uint_as_float(0xffffffffu);
    }
    __syncthreads();
    const float4 c = cand[l & (NW - 1)];
    u = __reduce_min_sync(0xffffffffu, __float_as_uint(c.x));
    const int ws = (int)((u / (uint32_t)(R * kDft)) & (NW - 1));  // warp w owns [R 64 w, R 64 (w + 1))
    ure = __shfl_sync(0xffffffffu, c.y, ws);
    uim = __shfl_sync(0xffffffffu, c.z, ws);
}

template <int kT, int kMinCtas>
__global__ void __launch_bounds__(kT, kMinCtas)
k_loop_planar(int iters, int blocks, float gamma, uint32_t *sums) {
    using L = Planar<kT>;
    constexpr int R = L::kR, NW = L::kNW;
    extern __shared__ __align__(128) unsigned char smem[];
    float *wre = reinterpret_cast<float *>(smem);
    float *wim = reinterpret_cast<float *>(smem + L::kPlane);
    float2 *A = reinterpret_cast<float2 *>(smem + L::kAOff);
    build_a(A);
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    for (int e = tid; e < L::kRows * kDft; e += kT) {
        const float2 a = A[(e / kDft) & (kDft - 1)], bq = A[e % kDft];
        wre[e] = a.x * bq.x - a.y * bq.y;
        wim[e] = a.x * bq.y + a.y * bq.x;
    }
    __syncthreads();
    const float gw = gamma / wre[0];
    uint32_t *smax = reinterpret_cast<uint32_t *>(smem + L::kSmaxOff);
    float4 *cand = reinterpret_cast<float4 *>(smem + L::kCandOff);
    float2 *dcl = reinterpret_cast<float2 *>(smem + L::kListOff);
    uint16_t *ul = reinterpret_cast<uint16_t *>(smem + L::kListOff + iters * 8);
    uint32_t sum = 0;
    for (int b = 0; b < blocks; ++b) {
        u64 rre[R], rim[R];
        init_spectrum<R>(blockIdx.x * blocks + b, rre, rim);
        u64 ndcr2 = 0ull, dci2 = 0ull, ndci2 = 0ull;
        int um = 0, un = 0;
        for (int it = 0; it < iters; ++it) {
            const int row = (R * w - um) & (kDft - 1), c = (l - un) & (kDft - 1);
            const float *pr0 = wre + row * kDft + c, *pr1 = wre + row * kDft + (c ^ 32);
            const float *pi0 = wim + row * kDft + c, *pi1 = wim + row * kDft + (c ^ 32);
            float mx = 0.f;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const u64 wr = pack2(pr0[r * kDft], pr1[r * kDft]);
                const u64 wi = pack2(pi0[r * kDft], pi1[r * kDft]);
                u64 a = fma2(wr, ndcr2, rre[r]);
                a = fma2(wi, dci2, a);
                u64 bb = fma2(wi, ndcr2, rim[r]);
                bb = fma2(wr, ndci2, bb);
                rre[r] = a;
                rim[r] = bb;
                const float2 e = unpack2(energy2(a, bb));
                mx = max3(mx, e.x, e.y);
            }
            uint32_t u;
            float ure, uim;
            select_planar<R, NW>(mx, rre, rim, smax, cand, u, ure, uim);
            const float dcr = ure * gw, dci = uim * gw;
            if (tid == 0) {
                dcl[it] = make_float2(dcr, dci);
                ul[it] = (uint16_t)u;
                sum = sum * 1000003u + u;
            }
            ndcr2 = pack2(-dcr, -dcr);
            dci2 = pack2(dci, dci);
            ndci2 = pack2(-dci, -dci);
            um = (int)((u >> 6) & 63u);
            un = (int)(u & 63u);
        }
        __syncthreads();
        if (tid == 0) sum += ul[iters - 1];
        __syncthreads();
    }
    if (tid == 0) sums[blockIdx.x] = sum;
}

typedef void (*LoopKernel)(int, int, float, uint32_t *);

struct LoopForm {
    LoopKernel k;
    int threads;
    int smem;
};

LoopForm loop_form(int variant, int iters) {
    const int w4 = lb_smem_bytes(iters);
    switch (variant) {
    case 0: return {k_loop<0>, kThreads, w4};
    case 1: return {k_loop<1>, kThreads, w4};
    case 2: return {k_loop<2>, kThreads, w4};
    case 3: return {k_loop<3>, kThreads, w4};
    case 4: return {k_loop<4>, kThreads, w4};
    case 5: return {k_loop<5>, kThreads, w4};
    case 6: return {k_loop<6>, kThreads, w4};
    case 7: return {k_loop<7>, kThreads, w4};
    case 8: return {k_loop<8>, kThreads, w4};
    case 9: return {k_loop_planar<256, 4>, 256, Planar<256>::smem_bytes(iters)};
    default: return {k_loop_planar<128, 4>, 128, Planar<128>::smem_bytes(iters)};
    }
}

}  // namespace

extern "C" int fse_loop_microbench(int device, int variant, int ctas_per_sm, int iters,
                                   int blocks_per_cta, double *ns_per_block_iter,
                                   uint32_t *checksum) {
    if (!ns_per_block_iter || !checksum || variant < 0 || variant > 10 || ctas_per_sm < 1 ||
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
    const LoopForm form = loop_form(variant, iters);
    int fit = 0;
    cudaError_t e = cudaFuncSetAttribute(form.k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         form.smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, form.k, form.threads, form.smem);
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
        form.k<<<grid, form.threads, form.smem>>>(iters, blocks_per_cta, 0.5f, sums);
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
