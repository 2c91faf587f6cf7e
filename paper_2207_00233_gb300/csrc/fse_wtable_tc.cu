// Weight-spectrum tables on the 5th-generation tensor cores (tcgen05): the
// 2-D DFT of a class pattern's 48x48 weights (Sec. 4: the DFT basis of the
// extrapolation; Eq. (2) weights) as two matrix products, with operands
// split into three TF32 parts and FP32 accumulators in tensor memory, which
// keeps the table at FP32 grade.
//
// One CTA of 128 threads per pattern.  With K-major operands (every row of
// an operand holds its K elements; D[i][j] = sum_k A[i][k] B[j][k]):
//   stage 1  D1[j][m] = sum_n B1[j][n] w[m][n]          M = 128, N = 48, K = 48
//            B1[j][n] = cos(2 pi j n / 64) (j < 64), -sin(2 pi (j - 64) n / 64)
//            so D1[j][m] = Re Y[m][j], D1[64 + j][m] = Im Y[m][j], the row DFT
//   stage 2  D2[j][km] = sum_k A2[j][k] C[km][k]         M = 128, N = 64, K = 96
//            C[km][k] = cos(2 pi km k / 64) (k < 48), sin(2 pi km (k - 48) / 64)
//            A2[j][k] = Re Y[k][j], Im Y[k - 48][j]            (j < 64)
//                       Im Y[k][j - 64], -Re Y[k - 48][j - 64] (j >= 64)
//            so D2[kn][km] = Re W[km][kn], D2[64 + kn][km] = Im W[km][kn].
// D2 is then made exactly conjugate-symmetric (W[-k] = conj W[k], the
// self-conjugate entries real), as the transform of real weights is: the
// iterations keep the residual's exact symmetry (and its exact ties) only if
// W has it.  The result is written in the W4 layout of the block kernels.
//
// Operands sit in shared memory without swizzle: 8-row x 16-byte core
// matrices, the core matrices of a row group adjacent along K (leading byte
// offset 128), row groups K * 32 bytes apart (stride byte offset).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/fse.h"
#include "fse_internal.h"

namespace fse {
namespace {

constexpr int kTcThreads = 128;
constexpr int kK1 = kArea;       // 48: stage-1 K (samples of a row)
constexpr int kK2 = 2 * kArea;   // 96: stage-2 K (rows, real and imaginary parts)
constexpr int kSbo1 = kK1 * 32;  // 1536
constexpr int kSbo2 = kK2 * 32;  // 3072

// Every operand is split into kParts TF32 parts, x = p0 + p1 + p2 (each
// rounded to TF32, |x - p0 - p1 - p2| <= 2^-33 |x|); a product keeps the six
// part products whose order is at most 2^-22 (p0 p0, p0 p1, p1 p0, p1 p1,
// p0 p2, p2 p0), so the tables are limited by the FP32 accumulation alone.
constexpr int kParts = 3;

// Shared-memory layout (bytes).  Stage 1 uses [0, 99 KB), stage 2 reuses
// [0, 144 KB) for A2 and keeps C at [144, 216 KB) from the start.
constexpr int kB1Bytes = 128 * kK1 * 4;              // 24576 per part
constexpr int kWOpBytes = kArea * kK1 * 4;           // 9216 per part
constexpr int kA2Bytes = 128 * kK2 * 4;              // 49152 per part
constexpr int kCBytes = kDft * kK2 * 4;              // 24576 per part
constexpr int kOffB1 = 0;                            // parts 0, 1, 2
constexpr int kOffW = kParts * kB1Bytes;             // parts 0, 1, 2
constexpr int kOffA2 = 0;                            // parts 0, 1, 2 (after stage 1)
constexpr int kOffC = kParts * kA2Bytes;             // parts 0, 1, 2
constexpr int kOffMisc = kOffC + kParts * kCBytes;   // mbarrier (8), tensor-memory address (4)
constexpr int kTcSmem = kOffMisc + 64;
static_assert(kOffW + kParts * kWOpBytes <= kOffC, "stage-1 operands overlap C");
static_assert(2 * kDft * kDft * 4 <= kOffC, "W planes overlap C");
static_assert(kTcSmem <= 227 * 1024, "shared memory of one CTA");
constexpr uint32_t kTmemCols = 128;                  // D1 at column 0, D2 at column 64

// Constant operand images (B1 then C, all parts each), as laid out in
// shared memory.
constexpr int kImageFloats = kParts * (kB1Bytes + kCBytes) / 4;

__device__ __forceinline__ int kmajor(int r, int k, int sbo) {
    return (r >> 3) * sbo + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}
// x rounded to the nearest TF32 value (10 stored mantissa bits; ties away
// from zero), so that the tensor core, which drops the low 13 bits of an
// FP32 operand, reads it exactly.  Each further part rounds what the
// earlier ones left: p1 = tf32(x - p0), p2 = tf32(x - p0 - p1).
__host__ __device__ inline float tf32_round(float x) {
#ifdef __CUDA_ARCH__
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
#endif
}

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// Shared-memory matrix descriptor: no swizzle, version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor: kind::tf32, FP32 accumulator, A and B K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 16 consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init1(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase with the given parity, at most limit_ns.
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity,
                                              unsigned long long limit_ns) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (now_ns() - t0 > limit_ns) return false;
    }
}
constexpr unsigned long long kMmaLimitNs = 1000000000ull;

// Writes the kParts TF32 parts of x at float offset o of parts `part_floats` apart.
__device__ __forceinline__ void put_parts(float *base, int part_floats, int o, float x) {
    float r = x;
#pragma unroll
    for (int q = 0; q < kParts; ++q) {
        const float p = tf32_round(r);
        base[q * part_floats + o] = p;
        r -= p;  // exact: p holds the leading bits of r
    }
}

// The six part products of one stage, K / 8 steps each, into the
// accumulator at tensor-memory address d; the smallest products first.
__device__ __forceinline__ void stage_mmas(uint32_t d, uint32_t a, uint32_t a_part,
                                           uint32_t b, uint32_t b_part, int ksteps, int sbo_a,
                                           int sbo_b, uint32_t idesc) {
    const int pa[6] = {1, 0, 2, 0, 1, 0}, pb[6] = {1, 2, 0, 1, 0, 0};
    uint32_t acc = 0u;
    for (int t = 0; t < 6; ++t)
        for (int k = 0; k < ksteps; ++k) {
            const uint32_t off = (uint32_t)k * 256u;  // 8 elements of K: two core matrices
            mma_tf32(d, sdesc(a + pa[t] * a_part + off, 128, sbo_a),
                     sdesc(b + pb[t] * b_part + off, 128, sbo_b), idesc, acc);
            acc = 1u;
        }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_wtable_tc(const int32_t *keys, const uint64_t *dst, float delta, const float *rho_tab,
            const float4 *image, int *error) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar = saddr(smem + kOffMisc);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffMisc + 8);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(tmem_slot)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) mbar_init1(bar);
    // constant operands: B1 at kOffB1 and C at kOffC, all parts
    {
        float4 *b1 = reinterpret_cast<float4 *>(smem + kOffB1);
        float4 *c = reinterpret_cast<float4 *>(smem + kOffC);
        for (int i = tid; i < kParts * kB1Bytes / 16; i += kTcThreads) b1[i] = image[i];
        for (int i = tid; i < kParts * kCBytes / 16; i += kTcThreads)
            c[i] = image[kParts * kB1Bytes / 16 + i];
    }
    // the weights of the pattern (Eq. (2)), K-major rows m, split
    {
        const int key = keys[blockIdx.x];
        float *wop = reinterpret_cast<float *>(smem + kOffW);
        for (int p = tid; p < kArea * kArea; p += kTcThreads) {
            const int m = p / kArea, n = p - m * kArea;
            const int cell = (m >> 4) * 3 + (n >> 4);
            float w = 0.f;
            if (cell != 4) {
                const int st = (key >> (2 * (cell < 4 ? cell : cell - 1))) & 3;
                if (st == 0) w = rho_tab[p];
                else if (st == 1) w = delta * rho_tab[p];
            }
            put_parts(wop, kWOpBytes / 4, kmajor(m, n, kSbo1) / 4, w);
        }
    }
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    // ---- stage 1: the row DFTs ----
    if (tid == 0) {
        stage_mmas(tmem, saddr(smem + kOffB1), kB1Bytes, saddr(smem + kOffW), kWOpBytes,
                   kK1 / 8, kSbo1, kSbo1, idesc_tf32(128, kArea));
        mma_commit(bar);
    }
    ok = __syncthreads_and(mbar_wait_for(bar, 0, kMmaLimitNs));
    if (ok) {
        fence_after_sync();
        // lane j = 32 warp + lane of D1: Re Y[m][j] (j < 64) or Im Y[m][j - 64]
        float v[48];
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float t[16];
            tmem_ld16(trow + 16 * c, t);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[16 * c + i] = t[i];
        }
        fence_before_sync();
        __syncthreads();  // stage-1 operands are no longer read (MMAs complete)
        // stage-2 A operand, K-major rows j: own row, columns 0..47, and the
        // partner row's columns 48..95
        const int j = tid;
        const int jp = j < kDft ? j + kDft : j - kDft;
        const float sgn = j < kDft ? -1.f : 1.f;
        float *aop = reinterpret_cast<float *>(smem + kOffA2);
#pragma unroll
        for (int m = 0; m < kArea; ++m) {
            put_parts(aop, kA2Bytes / 4, kmajor(j, m, kSbo2) / 4, v[m]);
            put_parts(aop, kA2Bytes / 4, kmajor(jp, kArea + m, kSbo2) / 4, sgn * v[m]);
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        // ---- stage 2: the column DFTs ----
        if (tid == 0) {
            stage_mmas(tmem + 64, saddr(smem + kOffA2), kA2Bytes, saddr(smem + kOffC), kCBytes,
                       kK2 / 8, kSbo2, kSbo2, idesc_tf32(128, kDft));
            mma_commit(bar);
        }
        ok = __syncthreads_and(mbar_wait_for(bar, 1, kMmaLimitNs));
        if (ok) {
            fence_after_sync();
            float u[64];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float t[16];
                tmem_ld16(trow + 64 + 16 * c, t);
#pragma unroll
                for (int i = 0; i < 16; ++i) u[16 * c + i] = t[i];
            }
            fence_before_sync();
            __syncthreads();  // stage-2 operands are no longer read
            // planes Re W[km][kn] (j < 64: kn = j) and Im W[km][kn] (kn = j - 64)
            float *pl = reinterpret_cast<float *>(smem);
#pragma unroll
            for (int km = 0; km < kDft; ++km) pl[(j >> 6) * kDft * kDft + km * kDft + (j & 63)] = u[km];
            __syncthreads();
            // exactly conjugate-symmetric W, written as W4 rows 0..70
            const float *pre = pl, *pim = pl + kDft * kDft;
            auto wv = [&](int km, int kn, float &re, float &im) {
                const int mk = (kDft - km) & (kDft - 1), mn = (kDft - kn) & (kDft - 1);
                const int lin = km * kDft + kn, mlin = mk * kDft + mn;
                if (lin <= mlin) {
                    re = pre[lin];
                    im = lin == mlin ? 0.f : pim[lin];
                } else {
                    re = pre[mlin];
                    im = -pim[mlin];
                }
            };
            float4 *out = reinterpret_cast<float4 *>(dst[blockIdx.x]);
            for (int e = tid; e < kW4Rows * kDft; e += kTcThreads) {
                const int row = (e / kDft) & (kDft - 1), c = e % kDft;
                float r0, i0, r1, i1;
                wv(row, c, r0, i0);
                wv(row, c ^ 32, r1, i1);
                out[e] = make_float4(r0, r1, i0, i1);
            }
        }
    }
    if (!ok) {
        if (tid == 0 && error) atomicExch(error, FSE_ETIMEDOUT);
        // products in flight land before the tensor memory is released
        mbar_wait_for(bar, 0, kMmaLimitNs);
        mbar_wait_for(bar, 1, kMmaLimitNs);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

// The constant operand images: B1 (128 x 48) and C (64 x 96), K-major, each
// as its three TF32 parts, in the shared-memory layout above.
void wtable_tc_image(std::vector<float> &img) {
    img.assign(kImageFloats, 0.f);
    auto kmaj = [](int r, int k, int sbo) {
        return (r >> 3) * sbo + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
    };
    const double step = 2.0 * 3.14159265358979323846 / kDft;
    auto put = [&](int base_bytes, int part_bytes, int r, int k, int sbo, double x) {
        // parts of the FP64 value (the constants are not limited to FP32)
        double rem = x;
        for (int q = 0; q < kParts; ++q) {
            const float pq = tf32_round((float)rem);
            img[(base_bytes + q * part_bytes + kmaj(r, k, sbo)) / 4] = pq;
            rem -= (double)pq;
        }
    };
    for (int j = 0; j < 128; ++j)
        for (int n = 0; n < kK1; ++n) {
            const int t = ((j & 63) * n) & (kDft - 1);
            put(0, kB1Bytes, j, n, kSbo1, j < kDft ? std::cos(step * t) : -std::sin(step * t));
        }
    for (int km = 0; km < kDft; ++km)
        for (int k = 0; k < kK2; ++k) {
            const int t = (km * (k % kArea)) & (kDft - 1);
            put(kParts * kB1Bytes, kCBytes, km, k, kSbo2,
                k < kArea ? std::cos(step * t) : std::sin(step * t));
        }
}
int wtable_tc_image_floats() { return kImageFloats; }

cudaError_t launch_wtables_tc(const int32_t *keys, const uint64_t *dst, int n, float delta,
                              const float *rho_tab, const float4 *image, int *error,
                              cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_wtable_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTcSmem);
    if (e != cudaSuccess) return e;
    k_wtable_tc<<<n, kTcThreads, kTcSmem, stream>>>(keys, dst, delta, rho_tab, image, error);
    return cudaGetLastError();
}

}  // namespace fse
