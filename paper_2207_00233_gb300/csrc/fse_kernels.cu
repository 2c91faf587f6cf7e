// sm_103a kernels of Frequency Selective Extrapolation (FSE) block
// concealment (Seiler & Kaup, Sec. 2 and Sec. 4) and the dispatch of the
// processing-order groups (Sec. 3, Algorithm 1).
//
// One CTA of 256 threads extrapolates one lost 16x16 block:
//   gather   48x48 area from the frame (luma and mask tiles by TMA bulk
//            tensor copies), sub-area classes, Eq. (2) weights
//   project  R_w = DFT64(w*f), W = DFT64(w)  (separable, real input; FP32
//            8-point split DFTs, or DFT-as-GEMM on the tensor cores)
//   iterate  K x { u = argmax |R_w|^2 ; dc = gamma R_w[u] / W[0] ;
//                  R_w[k] -= dc W[k - u] }       (Sec. 4, transform domain)
//   insert   Re sum dc_i phi_{u_i} on the lost samples of the block (Eq. (1))
//
// Thread (warp w, lane l) owns the 16 spectrum entries k_m = 8w + r
// (r = 0..7), k_n in {l, l + 32}; each (r) pair is held as two packed
// f32x2 registers (real parts, imaginary parts) so the update runs on the
// paired FP32 instructions of sm_100-class SMs.  W lives in shared memory
// in the W4 layout (see fse_internal.h): one 16-byte load per pair.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "../../include/fse.h"
#include "fse_internal.h"
#include "fse_iter.cuh"

namespace fse {
namespace {

using namespace fse::iter;  // packed FP32 pairs, W4 addressing, the loop body

// ---- TMA: bulk tensor copies completed on a shared-memory mbarrier ----------

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
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
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase with the given parity to complete; gives up after
// `limit_ns` nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
// 2-D tiled load of the box at (x, y) of `map` (x: innermost, in elements;
// out-of-range samples read as 0) into shared memory at `dst`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global memory into shared memory at `dst`, completing on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, uint64_t src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// A TMA copy that has not completed after this long is reported as an error.
constexpr unsigned long long kStageLimitNs = 2000000000ull;

// Copies a weight-spectrum table (kW4Bytes, W4 layout) into the W4 region
// with two bulk copies on the CTA's staging mbarrier (initialised, its next
// phase parity at kMbarOff + 8): wtable_begin (called by every thread after
// a barrier that ends the use of the region from kWTableSplit up) copies
// that upper part, wtable_finish (after a barrier that ends every use of the
// region) the part below and waits for both.  wtable_finish returns false
// on every thread when the copies did not complete within kStageLimitNs;
// they are then waited for once more, so that they do not land after the
// caller moves on.
constexpr int kWTableSplit = 18 * kDft * 16;  // W4 rows 0..17 below, 18..70 above
__device__ __forceinline__ void wtable_begin(unsigned char *smem, uint64_t table) {
    if (threadIdx.x == 0) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(smem + kMbarOff);
        // the region's earlier generic accesses come before the async copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, kW4Bytes);
        bulk_load((uint32_t)__cvta_generic_to_shared(smem + kWTableSplit), table + kWTableSplit,
                  kW4Bytes - kWTableSplit, bar);
    }
}
__device__ __forceinline__ bool wtable_finish(unsigned char *smem, uint64_t table) {
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(smem + kMbarOff);
    volatile uint32_t *phase = reinterpret_cast<volatile uint32_t *>(smem + kMbarOff + 8);
    const uint32_t ph = *phase;
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bulk_load((uint32_t)__cvta_generic_to_shared(smem), table, kWTableSplit, bar);
    }
    const bool ok = __syncthreads_and(mbar_wait(bar, ph, kStageLimitNs));
    if (!ok) mbar_wait(bar, ph, kStageLimitNs);
    if (threadIdx.x == 0) *phase = ph ^ 1u;
    return ok;
}

// ---- sources: where an area comes from and where its result goes -----------

// A block of a frame in a batch.  Classes follow Sec. 2: a lost sample of a
// block from an earlier group is R, of the block itself B_i, of a later
// group B_o.
struct FrameSrc {
    const FrameDesc &fd;
    int by, bx, self, gself;
    const unsigned char *stage;  // TMA-staged tiles of the area, or null

    __device__ FrameSrc(const FrameDesc &f, int block, const unsigned char *st = nullptr)
        : fd(f), by(block / f.bw), bx(block % f.bw), self(block), gself(f.gob[block]),
          stage(st) {}

    // The frame's fields, read once (the descriptor lives in global memory).
    struct Frame {
        int H, W, lb, bw, wstride;
        const int32_t *gob;
        const float *work;
    };
    __device__ __forceinline__ Frame frame() const {
        return Frame{fd.H, fd.W, fd.lb, fd.bw, fd.wstride, fd.gob, fd.work};
    }

    // Class and weight of the lost area sample at frame position (y, x):
    // R (an earlier-group block's concealed sample, read from the working
    // frame) or weight 0.
    __device__ __forceinline__ void classify_lost(const Frame &f, int y, int x, float rho,
                                                  float delta, float &w, float &v) const {
        const int cb = (y >> f.lb) * f.bw + (x >> f.lb);
        if (cb != self) {
            const int gc = f.gob[cb];
            if (gc >= 0 && gc < gself) {
                w = delta * rho;
                v = __ldcg(f.work + (size_t)y * f.wstride + x);
            }
        }
    }

    __device__ void gather(float *xt, float *wt, const float *rho_tab, float delta) const {
        const Frame f = frame();
        const int B = 1 << f.lb, M = B + 2 * kBorder;
        const int y0 = by * B - kBorder, x0 = bx * B - kBorder;
        if (stage) {
            // tiles start at column x0 rounded down to a multiple of 16
            const int dx = x0 - (x0 & ~15);
            const uint8_t *sl = stage;
            const uint8_t *sm = stage + (kStageMaskOff - kStageLumaOff);
            for (int p = threadIdx.x; p < kArea * kArea; p += kThreads) {
                const int m = p / kArea, n = p - m * kArea;
                const int y = y0 + m, x = x0 + n;
                float w = 0.f, v = 0.f;
                if (m < M && n < M && y >= 0 && y < f.H && x >= 0 && x < f.W) {
                    const int q = m * kStageCols + n + dx;
                    if (!sm[q]) {
                        w = rho_tab[p];
                        v = (float)sl[q];
                    } else {
                        classify_lost(f, y, x, rho_tab[p], delta, w, v);
                    }
                }
                xt[m * kTileStride + n] = w * v;
                wt[m * kTileStride + n] = w;
            }
            return;
        }
        const int stride = fd.stride;
        const uint8_t *mask = fd.mask, *luma = fd.luma;
        for (int p = threadIdx.x; p < kArea * kArea; p += kThreads) {
            const int m = p / kArea, n = p - m * kArea;
            const int y = y0 + m, x = x0 + n;
            float w = 0.f, v = 0.f;
            if (m < M && n < M && y >= 0 && y < f.H && x >= 0 && x < f.W) {
                const size_t q = (size_t)y * stride + x;
                if (!mask[q]) {
                    w = rho_tab[p];
                    v = (float)luma[q];
                } else {
                    classify_lost(f, y, x, rho_tab[p], delta, w, v);
                }
            }
            xt[m * kTileStride + n] = w * v;
            wt[m * kTileStride + n] = w;
        }
    }

    // Device address of the block's weight-spectrum table, 0 if it has none.
    __device__ __forceinline__ uint64_t table() const {
        const uint64_t *t = fd.wtab;
        return t ? t[self] : 0ull;
    }

    // Thread t holds the model value of sample (t / 16, t % 16) of the block.
    __device__ void store(float g) const {
        const int i = threadIdx.x >> 4, j = threadIdx.x & 15;
        const int lb = fd.lb;
        if (i >= (1 << lb) || j >= (1 << lb)) return;
        const int y = (by << lb) + i, x = (bx << lb) + j;
        if (y >= fd.H || x >= fd.W) return;
        const size_t q = (size_t)y * fd.stride + x;
        if (!fd.mask[q]) return;
        const float v = fminf(fmaxf(g, 0.f), 255.f);
        fd.work[(size_t)y * fd.wstride + x] = v;
        fd.out[q] = (uint8_t)__float2int_rn(v);
    }
};

// A pre-gathered area with explicit classes (inspection entry point).
struct AreaSrc {
    const float *f;
    const uint8_t *cls;
    float *g;
    int lb;

    __device__ void gather(float *xt, float *wt, const float *rho_tab, float delta) const {
        const int M = (1 << lb) + 2 * kBorder;
        for (int p = threadIdx.x; p < kArea * kArea; p += kThreads) {
            const int m = p / kArea, n = p - m * kArea;
            const int c = (m < M && n < M) ? cls[p] : 4;
            float w = 0.f;
            if (c == 0) w = rho_tab[p];
            else if (c == 1) w = delta * rho_tab[p];
            xt[m * kTileStride + n] = (w != 0.f) ? w * f[p] : 0.f;
            wt[m * kTileStride + n] = w;
        }
    }
    __device__ void store(float gv) const { g[threadIdx.x] = gv; }
    __device__ __forceinline__ uint64_t table() const { return 0ull; }
};

struct Trace {
    int32_t *u;   // [K] or null
    float *dc;    // [K][2] or null
    float *r;     // [64][64][2] or null
};

// Stage 2 of the projection for the entries of thread (w, l):
// X[k_m][k_n] = sum_m exp(-j 2 pi k_m m / 64) Y[m][k_n] for k_m = 8w + r and
// k_n in {l, l + 32}; column l + 32 comes from the conjugate of 32 - l.
// Lane 0 of each warp: entries of the real columns k_n = 0 and 32 for the
// warp's rows k_m = 8w + r, from xr (conjugated for k_m > 32).
__device__ __forceinline__ void real_cols(const float2 *xr, int w, int r, float &re0,
                                          float &im0, float &re1, float &im1) {
    const int k = 8 * w + r;
    const bool lo = k <= kDft / 2;
    const int kk = lo ? k : kDft - k;
    // loaded where used (the memory clobber keeps the compiler from hoisting
    // all sixteen loads, which would cost registers)
    float ar, ai, br, bi;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                 : "=f"(ar), "=f"(ai) : "r"(smem_addr(xr + kk)) : "memory");
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                 : "=f"(br), "=f"(bi) : "r"(smem_addr(xr + kHalfCols + kk)) : "memory");
    re0 = ar;
    im0 = lo ? ai : -ai;
    re1 = br;
    im1 = lo ? bi : -bi;
}

// Column DFT of the half spectrum y[48][33] (rows m, columns k_n) of one
// input, split as m = 8a + b (a < 6) and k_m = r + 8 q:
//   X[r + 8q][k_n] = sum_b e^{-j 2 pi b q / 8} T[b][r],
//   T[b][r] = e^{-j 2 pi r b / 64} sum_a y[8a + b][k_n] e^{-j 2 pi r a / 8}
// (the 64-point DFT as 8-point DFTs with twiddles; about a quarter of the
// multiply-adds of the direct sums, and shorter sums).
//
// Step 1: thread (w, l) computes T for b = w and column k_n = l and stores it
// as ts[k_n][8b + r] (complex; row stride kTsStride floats, so that the
// 16-byte loads of eight consecutive lanes fall into distinct banks).
//
// Columns k_n = 0 and 32 of a real input's spectrum are themselves
// conjugate-symmetric in k_m, so |R_w| ties exactly between k_m and -k_m
// there (as everywhere between k and -k before the first update).  The
// selection resolves exact ties to the smallest index, so the FP32 spectrum
// must keep the symmetry bit for bit: those two columns are summed directly
// for k_m <= 32 (xr[c][k_m]) and conjugated for k_m > 32.  Elsewhere the
// mirrored column repeats the partner entry's arithmetic exactly.
constexpr int kTsStride = 132;
constexpr int kXrOff = kHalfCols * kTsStride * 4;  // after ts of the x input
// (with a W table, step 2 reads only ts of w f and its real columns, below
// kWTableSplit = 18432 bytes: 17,952 bytes)
static_assert(kXrOff % 16 == 0 && kXrOff + 2 * 2 * kHalfCols * 8 <=
                                       kXTileOff + 2 * kArea * kTileStride * 4,
              "column-DFT scratch must fit the area tiles");
__device__ __forceinline__ void col_dft_step1(const float2 *y, float *ts, const float2 *tw,
                                              int b, int c) {
    float2 v[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) v[a] = y[(8 * a + b) * kHalfCols + c];
    float4 *out = reinterpret_cast<float4 *>(ts + c * kTsStride + 16 * b);
#pragma unroll
    for (int r = 0; r < 8; r += 2) {
        float t[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float zr = 0.f, zi = 0.f;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                // (c - j s) (v_r + j v_i)
                const float2 cs = tw[(8 * (r + h) * a) & (kDft - 1)];
                zr = fmaf(cs.x, v[a].x, fmaf(cs.y, v[a].y, zr));
                zi = fmaf(cs.x, v[a].y, fmaf(-cs.y, v[a].x, zi));
            }
            const float2 cs = tw[((r + h) * b) & (kDft - 1)];
            t[2 * h] = fmaf(cs.x, zr, cs.y * zi);
            t[2 * h + 1] = fmaf(cs.x, zi, -cs.y * zr);
        }
        out[r / 2] = make_float4(t[0], t[1], t[2], t[3]);
    }
}

// Step 2: thread (w, l) sums its rows k_m = 8w + r (q = w) of column l, and
// of column l + 32 through the conjugate symmetry of a real input's
// spectrum: X[k_m][l + 32] = conj(X[-k_m][32 - l]), where -k_m = r' + 8 q'
// with r' = -r mod 8 and q' = (8 - w) mod 8 for r = 0, 7 - w otherwise.
// Columns 0 and 32, rows 0..32: xr[c][k] (c = 0: k_n = 0, c = 1: k_n = 32)
// for the real column y[.][k_n] (its imaginary parts are exactly zero).
__device__ __forceinline__ void col_dft_real(const float2 *y, float2 *xr, const float2 *tw,
                                             int e) {
    const int c = e / kHalfCols, k = e - c * kHalfCols;
    const float2 *col = y + (c ? kHalfCols - 1 : 0);
    float re = 0.f, im = 0.f;
    for (int m = 0; m < kArea; ++m) {
        const float v = col[m * kHalfCols].x;
        const float2 cs = tw[(k * m) & (kDft - 1)];
        re = fmaf(v, cs.x, re);
        im = fmaf(-v, cs.y, im);
    }
    xr[e] = make_float2(re, im);
}

__device__ __forceinline__ void col_dft_step2(const float *ts, const float2 *tw, int w, int l,
                                              float (&ar)[8][2], float (&ai)[8][2]) {
    const float4 *dl = reinterpret_cast<const float4 *>(ts + l * kTsStride);
    const float4 *cl = reinterpret_cast<const float4 *>(ts + (32 - l) * kTsStride);
#pragma unroll
    for (int r = 0; r < 8; ++r) ar[r][0] = ai[r][0] = ar[r][1] = ai[r][1] = 0.f;
#pragma unroll 1
    for (int b = 0; b < 8; ++b) {
        const float2 cq = tw[(8 * w * b) & (kDft - 1)];        // e^{-j 2 pi b w / 8}
        const float2 cq7 = tw[(8 * (7 - w) * b) & (kDft - 1)];  // e^{-j 2 pi b (7 - w) / 8}
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // direct column: (c - j s) T[b][r], r = 2k, 2k + 1
            const float4 x = dl[4 * b + k];
            ar[2 * k][0] = fmaf(cq.x, x.x, fmaf(cq.y, x.y, ar[2 * k][0]));
            ai[2 * k][0] = fmaf(cq.x, x.y, fmaf(-cq.y, x.x, ai[2 * k][0]));
            ar[2 * k + 1][0] = fmaf(cq.x, x.z, fmaf(cq.y, x.w, ar[2 * k + 1][0]));
            ai[2 * k + 1][0] = fmaf(cq.x, x.w, fmaf(-cq.y, x.z, ai[2 * k + 1][0]));
            // mirrored column (conjugated at the end): T[b][r'] serves the
            // row r = -r' mod 8
            const float4 y = cl[4 * b + k];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rp = 2 * k + h, r = (8 - rp) & 7;
                const float tr = h ? y.z : y.x, ti = h ? y.w : y.y;
                if (r == 0) {  // e^{+j 2 pi b w / 8} = (c + j s)
                    ar[r][1] = fmaf(cq.x, tr, fmaf(-cq.y, ti, ar[r][1]));
                    ai[r][1] = fmaf(cq.x, ti, fmaf(cq.y, tr, ai[r][1]));
                } else {
                    ar[r][1] = fmaf(cq7.x, tr, fmaf(cq7.y, ti, ar[r][1]));
                    ai[r][1] = fmaf(cq7.x, ti, fmaf(-cq7.y, tr, ai[r][1]));
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) ai[r][1] = -ai[r][1];
}

// kW: also the spectrum of w (wre, wim and the real columns of W at
// kXrwOff); without it only R_w, for a block whose W comes from a table
// (the rows of w f take the same arithmetic either way).
// mid() runs on every thread after the barrier that ends the column DFTs'
// first step, when only the column intermediates of w f (below kWTableSplit
// bytes) are still to be read.
struct NoMid {
    __device__ void operator()() const {}
};
template <bool kW, class Mid = NoMid>
__device__ __forceinline__ void project_fp32(unsigned char *smem, const float2 *tw,
                                             u64 (&rre)[8], u64 (&rim)[8],
                                             float (&wre)[8][2], float (&wim)[8][2],
                                             Mid mid = Mid()) {
    constexpr int kRows = kW ? kYRows : kArea;  // rows of the row DFTs
    const float *xt = reinterpret_cast<const float *>(smem + kXTileOff);
    const float *wt = reinterpret_cast<const float *>(smem + kWTileOff);
    float2 *yx = reinterpret_cast<float2 *>(smem + kYxOff);
    float2 *yw = reinterpret_cast<float2 *>(smem + kYwOff);
    const int tid = threadIdx.x;

    // Row DFTs of the 96 real rows (w f, then w), split as n = 8a + b and
    // k_n = r + 8q like the column DFTs:
    //   Z[b][r] = sum_a v[8a + b] e^{-j 2 pi r a / 8}   (a < 6; real rows give
    //             Z[b][8 - r] = conj Z[b][r], so r = 0..4 are kept),
    //   Y[r + 8q] = sum_b e^{-j 2 pi (r + 8q) b / 64} Z[b][r].
    // Step A: item (b, row) (lanes: consecutive rows) stores Z[b][0], Z[b][4]
    // and Z[b][1..3] as eight planes zs[8b + slot][row].
    float *zs = reinterpret_cast<float *>(smem + kZsOff);
    for (int it = tid; it < 8 * kRows; it += kThreads) {
        const int bb = it / kRows, row = it - bb * kRows;
        const float *src = (row < kArea ? xt + row * kTileStride : wt + (row - kArea) * kTileStride);
        float v[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) v[a] = src[8 * a + bb];
        float *dst = zs + 8 * bb * kYRows + row;
        dst[0] = ((v[0] + v[1]) + (v[2] + v[3])) + (v[4] + v[5]);
        dst[kYRows] = ((v[0] - v[1]) + (v[2] - v[3])) + (v[4] - v[5]);
#pragma unroll
        for (int r = 1; r <= 3; ++r) {
            float zr = 0.f, zi = 0.f;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const float2 cs = tw[(8 * r * a) & (kDft - 1)];
                zr = fmaf(v[a], cs.x, zr);
                zi = fmaf(-v[a], cs.y, zi);
            }
            dst[2 * r * kYRows] = zr;
            dst[(2 * r + 1) * kYRows] = zi;
        }
    }
    __syncthreads();
    // Step B: item (r, row) (lanes: consecutive rows, r warp-uniform) sums
    // Y[r + 8q] for every q with r + 8q <= 32.
    for (int it = tid; it < 8 * kRows; it += kThreads) {
        const int r = it / kRows, row = it - r * kRows;
        const int rr = r <= 4 ? r : 8 - r;  // conj(Z[b][8 - r]) for r > 4
        const float sgn = r <= 4 ? 1.f : -1.f;
        float yr[5], yi[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) yr[q] = yi[q] = 0.f;
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) {
            const float *z = zs + 8 * bb * kYRows + row;
            float zr, zi;
            if (rr == 0) {
                zr = z[0];
                zi = 0.f;
            } else if (rr == 4) {
                zr = z[kYRows];
                zi = 0.f;
            } else {
                zr = z[2 * rr * kYRows];
                zi = sgn * z[(2 * rr + 1) * kYRows];
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if (r + 8 * q > kDft / 2) break;
                // (c - j s)(zr + j zi)
                const float2 cs = tw[((r + 8 * q) * bb) & (kDft - 1)];
                yr[q] = fmaf(cs.x, zr, fmaf(cs.y, zi, yr[q]));
                yi[q] = fmaf(cs.x, zi, fmaf(-cs.y, zr, yi[q]));
            }
        }
        float2 *y = (row < kArea ? yx + row * kHalfCols : yw + (row - kArea) * kHalfCols);
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (r + 8 * q <= kDft / 2) y[r + 8 * q] = make_float2(yr[q], yi[q]);
    }
    __syncthreads();

    const int w = tid >> 5, l = tid & 31;
    // Column DFTs: step 1 for both inputs (x into the free tile region, w
    // behind the half spectra), then step 2, x first.
    float *tsx = reinterpret_cast<float *>(smem + kXTileOff);
    float *tsw = reinterpret_cast<float *>(smem + kTswOff);
    float2 *xrx = reinterpret_cast<float2 *>(smem + kXrOff);
    col_dft_step1(yx, tsx, tw, w, l);
    if (kW) col_dft_step1(yw, tsw, tw, w, l);
    if (tid < 2 * kHalfCols) {
        col_dft_real(yx, xrx, tw, tid);
        if (kW) col_dft_real(yw, reinterpret_cast<float2 *>(smem + kXrwOff), tw, tid);
    }
    __syncthreads();
    mid();
    {
        float ar[8][2], ai[8][2];
        col_dft_step2(tsx, tw, w, l, ar, ai);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            rre[r] = pack2(ar[r][0], ar[r][1]);
            rim[r] = pack2(ai[r][0], ai[r][1]);
        }
    }
    if (l == 0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            float a, b, c, d;
            real_cols(xrx, w, r, a, b, c, d);
            rre[r] = pack2(a, c);
            rim[r] = pack2(b, d);
        }
    }
    // W's real columns are taken from xr when W is stored (store_w4): after
    // a selection of a self-conjugate index (the DC term, say) the residual
    // stays conjugate-symmetric only if W is.
    if (kW) col_dft_step2(tsw, tw, w, l, wre, wim);
}

// ---- projection on the tensor cores (warp-level mma.sync) --------------------

__device__ __forceinline__ uint32_t pk_bf16(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint32_t pk_f16(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ uint32_t cv_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// The two floats a bf16x2 register holds (exact).
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_f16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                        uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Per precision: K per mma instruction, and the operand registers of one
// fragment (x3 precisions carry a low part as well).
template <int P> struct Prec {
    static constexpr bool kTf32 = (P == FSE_PREC_TF32 || P == FSE_PREC_TF32X3);
    static constexpr int kStep = kTf32 ? 8 : 16;
    static constexpr bool kSplit = (P == FSE_PREC_BF16X3 || P == FSE_PREC_TF32X3);
};

// TF32 operand and, for the split type, the TF32 remainder.
template <int P>
__device__ __forceinline__ void cv_tf32_pair(float v, uint32_t &h, uint32_t &l) {
    h = cv_tf32(v);
    if (P == FSE_PREC_TF32X3) l = cv_tf32(v - __uint_as_float(h));
}

// An operand fragment: the 4 (A) or 2 (B) registers, plus the low parts.
struct FragA { uint32_t h[4], l[4]; };
struct FragB { uint32_t h[2], l[2]; };

// Pack two values that share a register, in the precision's type.
template <int P>
__device__ __forceinline__ void pack_pair(float v0, float v1, uint32_t &h, uint32_t &l) {
    if (P == FSE_PREC_FP16) {
        h = pk_f16(v0, v1);
    } else {
        h = pk_bf16(v0, v1);
        if (P == FSE_PREC_BF16X3) l = pk_bf16(v0 - bf_lo(h), v1 - bf_hi(h));
    }
}

// Fragment of a row-major A (16 x kStep) starting at (r0, k0) from a value
// functor A(row, k): the m16n8k16 / m16n8k8 register layouts.
template <int P, class FA>
__device__ __forceinline__ FragA load_a(FA A, int r0, int k0) {
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    FragA f;
    if (Prec<P>::kTf32) {
        cv_tf32_pair<P>(A(r0 + g, k0 + t), f.h[0], f.l[0]);
        cv_tf32_pair<P>(A(r0 + g + 8, k0 + t), f.h[1], f.l[1]);
        cv_tf32_pair<P>(A(r0 + g, k0 + t + 4), f.h[2], f.l[2]);
        cv_tf32_pair<P>(A(r0 + g + 8, k0 + t + 4), f.h[3], f.l[3]);
    } else {
        pack_pair<P>(A(r0 + g, k0 + 2 * t), A(r0 + g, k0 + 2 * t + 1), f.h[0], f.l[0]);
        pack_pair<P>(A(r0 + g + 8, k0 + 2 * t), A(r0 + g + 8, k0 + 2 * t + 1), f.h[1], f.l[1]);
        pack_pair<P>(A(r0 + g, k0 + 2 * t + 8), A(r0 + g, k0 + 2 * t + 9), f.h[2], f.l[2]);
        pack_pair<P>(A(r0 + g + 8, k0 + 2 * t + 8), A(r0 + g + 8, k0 + 2 * t + 9), f.h[3],
                     f.l[3]);
    }
    return f;
}

// Fragment of a (kStep x 8) B starting at (k0, c0) from a functor B(k, col).
template <int P, class FB>
__device__ __forceinline__ FragB load_b(FB B, int k0, int c0) {
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    FragB f;
    if (Prec<P>::kTf32) {
        cv_tf32_pair<P>(B(k0 + t, c0 + g), f.h[0], f.l[0]);
        cv_tf32_pair<P>(B(k0 + t + 4, c0 + g), f.h[1], f.l[1]);
    } else {
        pack_pair<P>(B(k0 + 2 * t, c0 + g), B(k0 + 2 * t + 1, c0 + g), f.h[0], f.l[0]);
        pack_pair<P>(B(k0 + 2 * t + 8, c0 + g), B(k0 + 2 * t + 9, c0 + g), f.h[1], f.l[1]);
    }
    return f;
}

template <int P>
__device__ __forceinline__ void mma_step(float (&d)[4], const FragA &a, const FragB &b) {
    if (Prec<P>::kTf32) {
        mma_tf32(d, a.h[0], a.h[1], a.h[2], a.h[3], b.h[0], b.h[1]);
        if (P == FSE_PREC_TF32X3) {
            mma_tf32(d, a.h[0], a.h[1], a.h[2], a.h[3], b.l[0], b.l[1]);
            mma_tf32(d, a.l[0], a.l[1], a.l[2], a.l[3], b.h[0], b.h[1]);
        }
    } else if (P == FSE_PREC_FP16) {
        mma_f16(d, a.h[0], a.h[1], a.h[2], a.h[3], b.h[0], b.h[1]);
    } else {
        mma_bf16(d, a.h[0], a.h[1], a.h[2], a.h[3], b.h[0], b.h[1]);
        if (P == FSE_PREC_BF16X3) {
            mma_bf16(d, a.h[0], a.h[1], a.h[2], a.h[3], b.l[0], b.l[1]);
            mma_bf16(d, a.l[0], a.l[1], a.l[2], a.l[3], b.h[0], b.h[1]);
        }
    }
}

// The constant operands: stage-1 B = [cos | -sin](k_n, n) and stage-2
// A = [cos | sin](k_m, m), from the exactly symmetric twiddle table.
struct DftB1 {
    const float2 *tw;
    __device__ float operator()(int k, int c) const {
        const int kn = c < 40 ? c : c - 40;
        if (kn >= kHalfCols) return 0.f;
        const float2 cs = tw[(kn * k) & (kDft - 1)];
        return c < 40 ? cs.x : -cs.y;
    }
};
struct DftA2 {
    const float2 *tw;
    __device__ float operator()(int km, int k) const {
        const float2 cs = tw[(km * (k < kArea ? k : k - kArea)) & (kDft - 1)];
        return k < kArea ? cs.x : cs.y;
    }
};

// Packed fragments of the constant operands, per precision:
//   stage-1 B: [10 n-tiles][K/kStep][32 lanes] -> uint4 (h0, h1, l0, l1)
//   stage-2 A: [4 m-tiles][96/kStep][32 lanes] -> 2 x uint4 (h0..h3, l0..l3)
template <int P> struct FragLayout {
    static constexpr int kS1 = kArea / Prec<P>::kStep;
    static constexpr int kS2 = 2 * kArea / Prec<P>::kStep;
    static constexpr int kB1 = 10 * kS1 * 32;       // uint4 entries
    static constexpr int kA2 = 4 * kS2 * 32 * 2;    // uint4 entries
};

template <int P>
__global__ void k_build_frags(const float2 *tw, uint4 *out) {
    using L = FragLayout<P>;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // one warp per fragment
    const int frag = i >> 5;
    if (frag < 10 * L::kS1) {
        const int nt = frag / L::kS1, ks = frag % L::kS1;
        const FragB f = load_b<P>(DftB1{tw}, ks * Prec<P>::kStep, nt * 8);
        out[i] = make_uint4(f.h[0], f.h[1], Prec<P>::kSplit ? f.l[0] : 0u,
                            Prec<P>::kSplit ? f.l[1] : 0u);
    } else if (frag < 10 * L::kS1 + 4 * L::kS2) {
        const int j = frag - 10 * L::kS1;
        const int mt = j / L::kS2, ks = j % L::kS2;
        const FragA f = load_a<P>(DftA2{tw}, mt * 16, ks * Prec<P>::kStep);
        const int base = L::kB1 + (j * 32 + (i & 31)) * 2;
        out[base] = make_uint4(f.h[0], f.h[1], f.h[2], f.h[3]);
        out[base + 1] = Prec<P>::kSplit ? make_uint4(f.l[0], f.l[1], f.l[2], f.l[3])
                                        : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Data operands: stage-1 A = the stacked tiles, stage-2 B from Y.
struct TileA1 {
    const float *xt, *wt;
    __device__ float operator()(int r, int k) const {
        return r < kArea ? xt[r * kTileStride + k] : wt[(r - kArea) * kTileStride + k];
    }
};
struct YB2 {
    const float *y;  // rows of this input's Y
    __device__ float operator()(int k, int c) const {
        if (k < kArea) return y[k * kYStride + c];
        const float *row = y + (k - kArea) * kYStride;
        return c < 40 ? row[c + 40] : -row[c - 40];
    }
};

template <int P>
__device__ __forceinline__ void project_mma(unsigned char *smem, const uint4 *frags,
                                            u64 (&rre)[8], u64 (&rim)[8],
                                            float (&wacc)[5][4]) {
    using L = FragLayout<P>;
    constexpr int KS = Prec<P>::kStep;
    const float *xt = reinterpret_cast<const float *>(smem + kXTileOff);
    const float *wt = reinterpret_cast<const float *>(smem + kWTileOff);
    float *y = reinterpret_cast<float *>(smem + kYOff);
    float2 *r0h = reinterpret_cast<float2 *>(smem + kR0Off);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;

    // Stage 1: Y (96 x 80) = tiles (96 x 48) x B1 (48 x 80); 6 x 10 tiles.
    for (int tile = w; tile < 60; tile += kWarps) {
        const int mt = tile / 10, nt = tile % 10;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < L::kS1; ++ks) {
            const FragA a = load_a<P>(TileA1{xt, wt}, mt * 16, ks * KS);
            const uint4 bv = frags[(nt * L::kS1 + ks) * 32 + lane];
            FragB b;
            b.h[0] = bv.x; b.h[1] = bv.y; b.l[0] = bv.z; b.l[1] = bv.w;
            mma_step<P>(d, a, b);
        }
        float *y0 = y + (mt * 16 + g) * kYStride + nt * 8 + 2 * t;
        y0[0] = d[0];
        y0[1] = d[1];
        y0[8 * kYStride] = d[2];
        y0[8 * kYStride + 1] = d[3];
    }
    __syncthreads();

    // Stage 2: warp w takes m-tile w & 3 and the n-tiles (w >> 2) * 5 .. +5 of
    // both inputs (x: R_w, then w: W).
    const int mt = w & 3, nt0 = (w >> 2) * 5;
    float xacc[5][4];
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) xacc[j][q] = wacc[j][q] = 0.f;
#pragma unroll 1
    for (int ks = 0; ks < L::kS2; ++ks) {
        const int fi = L::kB1 + ((mt * L::kS2 + ks) * 32 + lane) * 2;
        const uint4 ah = frags[fi], al = frags[fi + 1];
        FragA a;
        a.h[0] = ah.x; a.h[1] = ah.y; a.h[2] = ah.z; a.h[3] = ah.w;
        a.l[0] = al.x; a.l[1] = al.y; a.l[2] = al.z; a.l[3] = al.w;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            mma_step<P>(xacc[j], a, load_b<P>(YB2{y}, ks * KS, (nt0 + j) * 8));
            mma_step<P>(wacc[j], a, load_b<P>(YB2{y + kArea * kYStride}, ks * KS, (nt0 + j) * 8));
        }
    }
    // R_w, half spectrum, into the staging area (R0h[k_m][k_n], k_n <= 32).
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int km = mt * 16 + g + (q >> 1) * 8;
            const int c = (nt0 + j) * 8 + 2 * t + (q & 1);
            if (c < kHalfCols) r0h[km * kHalfCols + c].x = xacc[j][q];
            else if (c >= 40 && c < 40 + kHalfCols) r0h[km * kHalfCols + c - 40].y = xacc[j][q];
        }
    __syncthreads();
    // The entries this thread owns; k_n > 32 from the conjugate mirror.
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int km = 8 * w + r;
        const float2 a = r0h[km * kHalfCols + lane];
        float2 b;
        if (lane == 0) {
            b = r0h[km * kHalfCols + 32];
        } else {
            b = r0h[((kDft - km) & (kDft - 1)) * kHalfCols + 32 - lane];
            b.y = -b.y;
        }
        rre[r] = pack2(a.x, b.x);
        rim[r] = pack2(a.y, b.y);
    }
}

// W from the stage-2 fragments into the W4 layout (direct and conjugate
// mirror entries, repeated rows); the weight sum W[0] into *w0.
__device__ __forceinline__ void store_w4_frags(unsigned char *smem, const float (&wacc)[5][4],
                                               float *w0) {
    float *w4 = reinterpret_cast<float *>(smem);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int mt = w & 3, nt0 = (w >> 2) * 5;
    auto put = [&](int row, int col, int comp, float v) {
        // comp 0: real, 1: imaginary; slot .x/.z as the first member of
        // W4[row][col], .y/.w as the second member of W4[row][col ^ 32]
        const int a = (row * kDft + col) * 4 + 2 * comp;
        const int b = (row * kDft + (col ^ 32)) * 4 + 2 * comp + 1;
        w4[a] = v;
        w4[b] = v;
        if (row < kW4Rows - kDft) {
            w4[a + kDft * kDft * 4] = v;
            w4[b + kDft * kDft * 4] = v;
        }
    };
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int km = mt * 16 + g + (q >> 1) * 8;
            const int c = (nt0 + j) * 8 + 2 * t + (q & 1);
            const int comp = c < 40 ? 0 : 1;
            const int kn = c < 40 ? c : c - 40;
            if (kn >= kHalfCols) continue;
            const float v = wacc[j][q];
            put(km, kn, comp, v);
            if (kn != 0 && kn != 32)
                put((kDft - km) & (kDft - 1), kDft - kn, comp, comp ? -v : v);
            if (km == 0 && c == 0) *w0 = v;
        }
}

// Store the thread's W entries in the W4 layout (plus the repeated rows).
// Lane 0 then rewrites the real columns k_n = 0 and 32 from xr (exactly
// conjugate-symmetric in k_m; see col_dft_step1).
__device__ __forceinline__ void store_w4(unsigned char *smem, const float (&wre)[8][2],
                                         const float (&wim)[8][2], const float2 *xr) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    float4 *w4 = reinterpret_cast<float4 *>(smem);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int row = 8 * w + r;
        const float4 a = make_float4(wre[r][0], wre[r][1], wim[r][0], wim[r][1]);
        const float4 b = make_float4(wre[r][1], wre[r][0], wim[r][1], wim[r][0]);
        w4[row * kDft + l] = a;
        w4[row * kDft + l + 32] = b;
        if (row < kW4Rows - kDft) {
            w4[(row + kDft) * kDft + l] = a;
            w4[(row + kDft) * kDft + l + 32] = b;
        }
    }
    if (l != 0) return;
    for (int r = 0; r < 8; ++r) {
        const int row = 8 * w + r;
        float4 a;
        real_cols(xr, w, r, a.x, a.z, a.y, a.w);
        const float4 b = make_float4(a.y, a.x, a.w, a.z);
        w4[row * kDft] = a;
        w4[row * kDft + 32] = b;
        if (row < kW4Rows - kDft) {
            w4[(row + kDft) * kDft] = a;
            w4[(row + kDft) * kDft + 32] = b;
        }
    }
}

static_assert(kXrOff + 2 * kHalfCols * 8 <= kWTableSplit,
              "the x-only second column step reads below the table's upper part");

// Thread 0's clock at phase boundary p of the current block (kept in shared
// memory; the instrumented persistent executor copies them out).  Phases:
// 0 claimed, 1 dependencies ready, 2 area staged, 3 gathered, 4 projected
// (W in place), 5 iterated, 6 synthesised, 7 stored and released.  The
// stamps at 3, 4 and 5 are taken in every instantiation: three shared
// stores per block, and with them the persistent kernel measured 1-2%
// faster on the 16-frame 1080p batch (A/B builds; same registers and
// spills: the code around the iteration loop is scheduled differently).
// The others, and the copy-out, belong to the instrumented executor only.
template <bool kOn>
__device__ __forceinline__ void phase_stamp(unsigned char *smem, int p) {
    if (kOn && threadIdx.x == 0) {
        uint32_t t;
        asm volatile("mov.u32 %0, %%clock;" : "=r"(t));
        reinterpret_cast<volatile uint32_t *>(smem + kStampOff)[p] = t;
    }
}

// The full per-block computation.  Returns the model value of this thread's
// sample of the centre block (unclamped).
template <int P, bool kTrace, bool kStamps = false, class Src>
__device__ __forceinline__ float run_block(const Src &src, const KParams &kp,
                                           const float *rho_tab, const float2 *tw_g,
                                           unsigned char *smem, const Trace &tr) {
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    float2 *tw = reinterpret_cast<float2 *>(smem + kTwOff);
    uint32_t *smax = reinterpret_cast<uint32_t *>(smem + kRedOff);
    uint4 *slot = reinterpret_cast<uint4 *>(smem + kRedOff + 32);  // the published step
    float *misc = reinterpret_cast<float *>(smem + kRedOff + 32 + 128);
    float2 *dcl = reinterpret_cast<float2 *>(smem + kListOff);
    uint16_t *ul = reinterpret_cast<uint16_t *>(smem + kListOff + kp.iters * 8);

    if (tid < kDft) tw[tid] = tw_g[tid];
    src.gather(reinterpret_cast<float *>(smem + kXTileOff),
               reinterpret_cast<float *>(smem + kWTileOff), rho_tab, kp.delta);
    __syncthreads();
    phase_stamp<true>(smem, 3);

    u64 rre[8], rim[8];
    if (P == FSE_PREC_FP32) {
        float wre[8][2], wim[8][2];
        // W from the block's table (bulk copy; needs the staging mbarrier,
        // which exists when shared memory starts 128-byte aligned) or
        // computed here
        const uint64_t wtab = ((smem_addr(smem) & 127u) == 0u) ? src.table() : 0ull;
        if (wtab) {
            // the upper part of the table is copied in while the column
            // DFTs' second step still reads the lower part of the region
            project_fp32<false>(smem, tw, rre, rim, wre, wim,
                                [&] { wtable_begin(smem, wtab); });
            __syncthreads();  // all reads of the projection scratch are done
            if (!wtable_finish(smem, wtab) && tid == 0 && kp.error)
                atomicExch(kp.error, FSE_ETIMEDOUT);
            if (tid == 0) misc[0] = reinterpret_cast<const float4 *>(smem)[0].x;  // W[0]
        } else {
            project_fp32<true>(smem, tw, rre, rim, wre, wim);
            __syncthreads();  // all reads of the stage-1 scratch are done
            const float2 *xrw = reinterpret_cast<const float2 *>(smem + kXrwOff);
            store_w4(smem, wre, wim, xrw);
            if (tid == 0) misc[0] = xrw[0].x;  // W[0] = sum of the weights
        }
    } else {
        float wacc[5][4];
        project_mma<P>(smem, kp.frags, rre, rim, wacc);
        __syncthreads();  // all reads of the projection scratch are done
        store_w4_frags(smem, wacc, misc);
    }
    __syncthreads();

    phase_stamp<true>(smem, 4);
    const float W0 = misc[0];
    const int K = (W0 > 0.f) ? kp.iters : 0;
    const float gw = kp.gamma / fmaxf(W0, 1e-30f);
    const uint32_t w4addr = smem_addr(smem);

    // Sec. 4 iterations.  Per iteration: the update with the previous
    // coefficient (none in the first pass) and every thread's maximum
    // energy; then the selection: the warp maxima meet at a barrier, the
    // smallest warp holding the block maximum searches its entries for the
    // smallest index, and its lane that holds it computes dc = gamma R_w[u] /
    // W[0], appends (dc, u) to the lists and publishes the update step,
    // which every thread reads after a second barrier.  (The loop
    // microbenchmark compares this form with the alternatives.)
    const uint32_t w8k = (uint32_t)(8 * w) << 10, l16 = (uint32_t)l << 4;
    Step st{0ull, 0ull, 0ull, 0u, 0u};  // first pass: dc = 0
    for (int it = 0; it < K; ++it) {
        const uint32_t wb = w4_addr_of(w4addr, w8k, l16, st);
        const float tmx = update_and_max(wb, st.ndcr2, st.dci2, st.ndci2, rre, rim);
        select_named_warp<false>(tmx, rre, rim, gw, it, smax, slot, dcl, ul, st);
    }
    if (kTrace && tr.r) {  // residual after the last update (inspection only)
        if (K > 0)
            update_and_max(w4_addr_of(w4addr, w8k, l16, st), st.ndcr2, st.dci2, st.ndci2, rre,
                           rim);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float2 re = unpack2(rre[r]), im = unpack2(rim[r]);
            const int km = 8 * w + r;
            tr.r[(km * kDft + l) * 2] = re.x;
            tr.r[(km * kDft + l) * 2 + 1] = im.x;
            tr.r[(km * kDft + l + 32) * 2] = re.y;
            tr.r[(km * kDft + l + 32) * 2 + 1] = im.y;
        }
    }
    __syncthreads();  // list complete
    phase_stamp<true>(smem, 5);
    if (kTrace && (tr.u || tr.dc)) {
        for (int it = tid; it < kp.iters; it += kThreads) {
            if (tr.u) tr.u[it] = (it < K) ? (int32_t)ul[it] : -1;
            if (tr.dc) {
                const float2 d = (it < K) ? dcl[it] : make_float2(0.f, 0.f);
                tr.dc[2 * it] = d.x;
                tr.dc[2 * it + 1] = d.y;
            }
        }
    }

    // Eq. (1) on the centre block: Re sum_it dc_it exp(+j 2 pi (u_m m + u_n n)/64)
    // with m = 16 + i, n = 16 + j.  The exponential factorises: with
    // P[it][i] = dc_it exp(+j 2 pi u_m m / 64) and E[it][j] = exp(+j 2 pi u_n n / 64),
    // g[i][j] = sum_it (Re P Re E - Im P Im E), a real product of a 16 x 2K and
    // a 2K x 16 matrix.  Per chunk of iterations the tables are built in the
    // (now free) W4 region; warp s takes the iterations it = s mod 8, each of
    // its threads a 2 x 4 tile of samples (rows i0, i0 + 1; columns j0..j0 + 3)
    // in packed f32x2 multiply-adds; the eight partial tiles of a sample are
    // then added in warp order.
    u64 *ptab = reinterpret_cast<u64 *>(smem);  // [it][i]: (Re P, Re P), (-Im P, -Im P)
    float *etab = reinterpret_cast<float *>(smem + kSynChunk * 16 * 16);  // [it]: Re E[16], Im E[16]
    const int tq = tid & 31, i0 = 2 * (tq >> 2), j0 = 4 * (tq & 3);
    u64 acc00 = 0ull, acc01 = 0ull, acc10 = 0ull, acc11 = 0ull;  // acc[row][column pair]
    for (int c0 = 0; c0 < K; c0 += kSynChunk) {
        const int nc = min(kSynChunk, K - c0);
        // thread (it, q) builds P[it][q] and E[it][q]: no divergent halves,
        // and two independent table lookups per entry
#pragma unroll 2
        for (int e = tid; e < nc * 16; e += kThreads) {
            const int it = e >> 4, q = e & 15;
            const int u = ul[c0 + it];
            const float2 d = dcl[c0 + it];
            const float2 cm = tw[((u >> 6) * (kBorder + q)) & (kDft - 1)];
            const float2 cn = tw[((u & 63) * (kBorder + q)) & (kDft - 1)];
            const float pr = fmaf(d.x, cm.x, -d.y * cm.y), pim = fmaf(d.x, cm.y, d.y * cm.x);
            st_shared_pair(smem_addr(ptab + (it * 16 + q) * 2), pack2(pr, pr), pack2(-pim, -pim));
            etab[it * 32 + q] = cn.x;
            etab[it * 32 + 16 + q] = cn.y;
        }
        __syncthreads();
        const uint32_t pbase = smem_addr(ptab) + (uint32_t)i0 * 16u;
        const uint32_t ebase = smem_addr(etab) + (uint32_t)j0 * 4u;
        for (int it = w; it < nc; it += kWarps) {
            u64 p0r, p0i, p1r, p1i, er0, er1, ei0, ei1;
            lds_pair(pbase + (uint32_t)it * 256u, p0r, p0i);
            lds_pair(pbase + (uint32_t)it * 256u + 16u, p1r, p1i);
            lds_pair(ebase + (uint32_t)it * 128u, er0, er1);
            lds_pair(ebase + (uint32_t)it * 128u + 64u, ei0, ei1);
            acc00 = fma2(p0i, ei0, fma2(p0r, er0, acc00));
            acc01 = fma2(p0i, ei1, fma2(p0r, er1, acc01));
            acc10 = fma2(p1i, ei0, fma2(p1r, er0, acc10));
            acc11 = fma2(p1i, ei1, fma2(p1r, er1, acc11));
        }
        __syncthreads();
    }
    float *part = reinterpret_cast<float *>(smem + kSynPartOff);  // [warp][i][j]
    st_shared_pair(smem_addr(part + w * 256 + i0 * 16 + j0), acc00, acc01);
    st_shared_pair(smem_addr(part + w * 256 + (i0 + 1) * 16 + j0), acc10, acc11);
    __syncthreads();
    float g = part[tid];
#pragma unroll
    for (int s2 = 1; s2 < kWarps; ++s2) g += part[s2 * 256 + tid];
    return g;
}

// ---- kernels -------------------------------------------------------------------

// Selection trace of a frame block (inspection option): the K selected
// indices from the shared list, -1 when the area had no support.  Runs after
// run_block, whose last barrier completed the list.
__device__ __forceinline__ void write_frame_trace(const FrameDesc &fd, int block,
                                                  const KParams &kp, const unsigned char *smem) {
    if (!fd.trace) return;
    const float W0 = reinterpret_cast<const float *>(smem + kRedOff + 32 + 128)[0];
    const uint16_t *ul = reinterpret_cast<const uint16_t *>(smem + kListOff + kp.iters * 8);
    int16_t *t = fd.trace + (size_t)block * kp.iters;
    for (int it = threadIdx.x; it < kp.iters; it += kThreads)
        t[it] = (W0 > 0.f) ? (int16_t)ul[it] : (int16_t)-1;
}

// The CTA's staging mbarrier and the parity of its next phase (shared, so
// that no register carries it through the iterations).
__device__ __forceinline__ void stage_init(unsigned char *smem) {
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(smem + kMbarOff), 1);
        *reinterpret_cast<uint32_t *>(smem + kMbarOff + 8) = 0u;
    }
}

// Stages the luma and mask tiles of the area of `block` with two TMA copies
// completing on the CTA's mbarrier.  Returns false on every
// thread when the copies did not complete within kStageLimitNs; the caller
// then leaves the kernel.
__device__ __forceinline__ bool stage_area(const FrameDesc &fd, int block, unsigned char *smem) {
    const uint32_t bar = smem_addr(smem + kMbarOff);
    volatile uint32_t *phase = reinterpret_cast<volatile uint32_t *>(smem + kMbarOff + 8);
    const uint32_t ph = *phase;
    if (threadIdx.x == 0) {
        const int B = 1 << fd.lb, by = block / fd.bw, bx = block - by * fd.bw;
        const int y0 = by * B - kBorder, xs = (bx * B - kBorder) & ~15;
        const unsigned char *maps = static_cast<const unsigned char *>(fd.tmaps);
        // Order the CTA's earlier generic accesses to the staging region
        // (previous block) before the copies.  (The kernel never writes the
        // staged samples that it uses: an `out` aliasing `luma` changes lost
        // samples only, whose luma is not read.)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, kStageBytes);
        tma_load_2d(smem_addr(smem + kStageLumaOff), maps, xs, y0, bar);
        tma_load_2d(smem_addr(smem + kStageMaskOff), maps + kTensorMapBytes, xs, y0, bar);
    }
    const bool ok = __syncthreads_and(mbar_wait(bar, ph, kStageLimitNs));
    if (!ok) mbar_wait(bar, ph, kStageLimitNs);  // copies in flight land before leaving
    if (threadIdx.x == 0) *phase = ph ^ 1u;      // every thread has read it
    return ok;
}

// Shared memory of the block kernels starts 128-byte aligned (TMA
// destinations); checked at run time, frames fall back to plain loads if not.
__device__ __forceinline__ bool stage_capable(const unsigned char *smem) {
    return (smem_addr(smem) & 127u) == 0;
}

template <int P>
__global__ void __launch_bounds__(kThreads, 3)
k_group(const FrameDesc *frames, const int2 *items, KParams kp, const float *rho_tab,
        const float2 *tw_tab) {
    extern __shared__ __align__(128) unsigned char smem[];
    float g;
    {
        const int2 item = items[blockIdx.x];
        const FrameDesc &fd = frames[item.x];
        const unsigned char *stage = nullptr;
        if (stage_capable(smem)) stage_init(smem);  // staging and table copies
        __syncthreads();
        if (fd.tmaps && kp.error && stage_capable(smem)) {
            if (!stage_area(fd, item.y, smem)) {
                if (threadIdx.x == 0) atomicExch(kp.error, FSE_ETIMEDOUT);
                return;
            }
            stage = smem + kStageLumaOff;
        }
        const FrameSrc src(fd, item.y, stage);
        g = run_block<P, false>(src, kp, rho_tab, tw_tab, smem, Trace{nullptr, nullptr, nullptr});
    }
    // Reload the item instead of keeping it live through the iterations.
    asm volatile("" ::: "memory");
    const int2 item = items[blockIdx.x];
    const FrameSrc src(frames[item.x], item.y);
    src.store(g);
    write_frame_trace(frames[item.x], item.y, kp, smem);
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Warp 0 waits, with bounded polling, for the completion flags of the
// earlier-group lost blocks whose samples lie in the area of `block`
// (+-16/B blocks).  Returns false when a wait gave up or another CTA
// reported an error.
__device__ __forceinline__ bool wait_area(const FrameDesc &fd, int block, bool stuck,
                                          const WorkQueue &q) {
    const int lane = threadIdx.x & 31;
    const int rad = kBorder >> fd.lb, side = 2 * rad + 1;
    const int by = block / fd.bw, bx = block - by * fd.bw;
    const int gself = fd.gob[block];
    bool ok = true;
    for (int p = lane; p < side * side + (stuck ? 1 : 0) && ok; p += 32) {
        int c;
        if (p == side * side) {
            c = block;  // test hook: a flag nothing sets before this wait ends
        } else {
            const int ny = by + p / side - rad, nx = bx + p % side - rad;
            if (ny < 0 || ny >= fd.bh || nx < 0 || nx >= fd.bw || (ny == by && nx == bx))
                continue;
            c = ny * fd.bw + nx;
            const int gc = fd.gob[c];
            if (gc < 0 || gc >= gself) continue;
        }
        long long spins = 0;
        while (ld_acquire_u32(fd.done + c) == 0u) {
            if (++spins > q.spin_limit) {
                atomicExch(q.error, FSE_ETIMEDOUT);
                ok = false;
                break;
            }
            if ((spins & 255) == 0 && *(volatile int *)q.error) {
                ok = false;
                break;
            }
            __nanosleep(200);
        }
    }
    return __all_sync(0xffffffffu, ok);
}

template <int P, bool kStamps>
__global__ void __launch_bounds__(kThreads, 3)
k_persistent(const FrameDesc *frames, WorkQueue q, KParams kp, const float *rho_tab,
             const float2 *tw_tab) {
    extern __shared__ __align__(128) unsigned char smem[];
    // claimed item and wait result, beside the mbarrier (no static shared
    // memory, so that the dynamic region starts at the window's base)
    int &s_item = *reinterpret_cast<int *>(smem + kMbarOff + 12);
    int &s_ok = *reinterpret_cast<int *>(smem + kMbarOff + 16);
    if (stage_capable(smem)) stage_init(smem);  // made visible by the first barrier below
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(q.head, 1);
        __syncthreads();
        const int i = s_item;
        if (i >= q.n) break;
        phase_stamp<kStamps>(smem, 0);
        if (threadIdx.x < 32) {
            const int2 item = q.items[i];
            const bool ok = wait_area(frames[item.x], item.y, i == q.stuck_item, q);
            if (threadIdx.x == 0) s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        phase_stamp<kStamps>(smem, 1);
        float g;
        {
            const int2 item = q.items[i];
            const FrameDesc &fd = frames[item.x];
            const unsigned char *stage = nullptr;
            if (fd.tmaps && stage_capable(smem)) {
                if (!stage_area(fd, item.y, smem)) {
                    if (threadIdx.x == 0) atomicExch(q.error, FSE_ETIMEDOUT);
                    break;
                }
                stage = smem + kStageLumaOff;
            }
            phase_stamp<kStamps>(smem, 2);
            const FrameSrc src(fd, item.y, stage);
            g = run_block<P, false, kStamps>(src, kp, rho_tab, tw_tab, smem,
                                             Trace{nullptr, nullptr, nullptr});
            phase_stamp<kStamps>(smem, 6);
        }
        // Reload the item instead of keeping it live through the iterations.
        asm volatile("" ::: "memory");
        const int2 item = q.items[s_item];
        const FrameSrc src(frames[item.x], item.y);
        src.store(g);
        write_frame_trace(frames[item.x], item.y, kp, smem);
        // Every thread's samples precede the barrier; thread 0's fence is
        // cumulative over what the barrier ordered before it, so one fence
        // and the release store publish the whole block at GPU scope.
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u32(frames[item.x].done + item.y, 1u);
            if (kStamps && kp.clocks) {
                phase_stamp<kStamps>(smem, 7);
                const volatile uint32_t *st =
                    reinterpret_cast<const volatile uint32_t *>(smem + kStampOff);
                uint32_t *dst = kp.clocks + (size_t)s_item * kPhaseStamps;
                for (int k = 0; k < kPhaseStamps; ++k) dst[k] = st[k];
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(kThreads, 3)
k_areas(const float *area_f, const uint8_t *area_cls, KParams kp, const float *rho_tab,
        const float2 *tw_tab, float *g_out, int32_t *u_out, float *dc_out, float *r_out) {
    extern __shared__ __align__(128) unsigned char smem[];
    const size_t a = blockIdx.x;
    const AreaSrc src{area_f + a * kArea * kArea, area_cls + a * kArea * kArea,
                      g_out + a * kBlock * kBlock, kp.lb};
    const Trace tr{u_out ? u_out + a * kp.iters : nullptr,
                   dc_out ? dc_out + a * kp.iters * 2 : nullptr,
                   r_out ? r_out + a * kDft * kDft * 2 : nullptr};
    const float g = run_block<P, true>(src, kp, rho_tab, tw_tab, smem, tr);
    src.store(g);
}

// Weight-spectrum tables: one CTA per key builds the 48x48 weights of the
// class pattern the key encodes (Eq. (2): rho^dist on A, delta rho^dist on
// R, 0 on B_i, B_o and outside), takes its DFT with the same FP32 split DFTs
// as the per-block kernels (so a table equals the W a block would compute)
// and writes the W4 region to the table.
__global__ void __launch_bounds__(kThreads, 3)
k_wtable(const int32_t *keys, const uint64_t *dst, float delta, const float *rho_tab,
         const float2 *tw_tab) {
    extern __shared__ __align__(128) unsigned char smem[];
    float2 *tw = reinterpret_cast<float2 *>(smem + kTwOff);
    if (threadIdx.x < kDft) tw[threadIdx.x] = tw_tab[threadIdx.x];
    const int key = keys[blockIdx.x];
    float *xt = reinterpret_cast<float *>(smem + kXTileOff);
    float *wt = reinterpret_cast<float *>(smem + kWTileOff);
    for (int p = threadIdx.x; p < kArea * kArea; p += kThreads) {
        const int m = p / kArea, n = p - m * kArea;
        const int cell = (m >> 4) * 3 + (n >> 4);  // 3x3 cells of 16x16, centre 4
        float w = 0.f;
        if (cell != 4) {
            const int st = (key >> (2 * (cell < 4 ? cell : cell - 1))) & 3;
            if (st == 0) w = rho_tab[p];
            else if (st == 1) w = delta * rho_tab[p];
        }
        xt[m * kTileStride + n] = 0.f;
        wt[m * kTileStride + n] = w;
    }
    __syncthreads();
    u64 rre[8], rim[8];
    float wre[8][2], wim[8][2];
    project_fp32<true>(smem, tw, rre, rim, wre, wim);
    __syncthreads();
    store_w4(smem, wre, wim, reinterpret_cast<const float2 *>(smem + kXrwOff));
    __syncthreads();
    uint4 *out = reinterpret_cast<uint4 *>(dst[blockIdx.x]);
    const uint4 *src = reinterpret_cast<const uint4 *>(smem);
    for (int i = threadIdx.x; i < kW4Bytes / 16; i += kThreads) out[i] = src[i];
}

// Block-loss map: one thread per (frame, sample row, block column) scans the
// 16 samples of that block row.
__global__ void k_block_loss(const FrameDesc *frames, uint8_t *lost, uint8_t *part,
                             const int *lost_off) {
    const FrameDesc &fd = frames[blockIdx.y];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= fd.H * fd.bw) return;
    const int y = idx / fd.bw, bx = idx - y * fd.bw;
    const int B = 1 << fd.lb;
    const uint8_t *row = fd.mask + (size_t)y * fd.stride + bx * B;
    const int n = min(B, fd.W - bx * B);
    int any = 0, all = 1;
    for (int i = 0; i < n; ++i) {
        any |= row[i];
        all &= row[i] != 0;
    }
    const int b = lost_off[blockIdx.y] + (y >> fd.lb) * fd.bw + bx;
    if (any) lost[b] = 1;
    if (part && !all) part[b] = 1;
}

}  // namespace

// ---- launchers ------------------------------------------------------------------

// Calls f with the precision as a compile-time constant.
template <class F>
static cudaError_t with_precision(int precision, F f) {
    switch (precision) {
    case FSE_PREC_FP32: return f(std::integral_constant<int, FSE_PREC_FP32>());
    case FSE_PREC_TF32: return f(std::integral_constant<int, FSE_PREC_TF32>());
    case FSE_PREC_BF16: return f(std::integral_constant<int, FSE_PREC_BF16>());
    case FSE_PREC_FP16: return f(std::integral_constant<int, FSE_PREC_FP16>());
    case FSE_PREC_BF16X3: return f(std::integral_constant<int, FSE_PREC_BF16X3>());
    case FSE_PREC_TF32X3: return f(std::integral_constant<int, FSE_PREC_TF32X3>());
    default: return cudaErrorInvalidValue;
    }
}

// The dynamic shared-memory limit is a per-device (per-context) attribute
// of each kernel: it is set once per device and precision, under a lock
// (the serving, host-batch and caller threads all launch); bit d of
// g_attr_done[precision] records device d.  Devices beyond 63 set it on
// every launch.
static std::atomic<uint64_t> g_attr_done[6];
static std::mutex g_attr_mu;

static cudaError_t ensure_attrs(int precision) {
    if (precision < 0 || precision > 5) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (g_attr_done[precision].load(std::memory_order_acquire) & bit)) return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (bit && (g_attr_done[precision].load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const int max_smem = smem_bytes(FSE_MAX_ITERS);
    e = with_precision(precision, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        cudaError_t r = cudaFuncSetAttribute(k_group<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             max_smem);
        if (r != cudaSuccess) return r;
        r = cudaFuncSetAttribute(k_persistent<P, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (r != cudaSuccess) return r;
        if (P == FSE_PREC_FP32) {
            r = cudaFuncSetAttribute(k_persistent<FSE_PREC_FP32, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
            if (r != cudaSuccess) return r;
        }
        r = cudaFuncSetAttribute(k_areas<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem);
        if (r != cudaSuccess) return r;
        return cudaFuncSetAttribute(k_wtable, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem_bytes(0));
    });
    if (e == cudaSuccess && bit) g_attr_done[precision].fetch_or(bit, std::memory_order_release);
    return e;
}

bool precision_supported(int precision) { return precision >= 0 && precision <= 5; }

size_t frag_bytes(int precision) {
    size_t n = 0;
    with_precision(precision, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        n = (size_t)(FragLayout<P>::kB1 + FragLayout<P>::kA2) * sizeof(uint4);
        return cudaSuccess;
    });
    return precision == FSE_PREC_FP32 ? 0 : n;
}

cudaError_t launch_build_frags(int precision, const float2 *tw, uint4 *out, cudaStream_t stream) {
    if (precision == FSE_PREC_FP32) return cudaSuccess;
    return with_precision(precision, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        using L = FragLayout<P>;
        const int warps = 10 * L::kS1 + 4 * L::kS2;
        k_build_frags<P><<<(warps * 32 + 255) / 256, 256, 0, stream>>>(tw, out);
        return cudaGetLastError();
    });
}

int max_resident_ctas(int iters) {
    if (ensure_attrs(FSE_PREC_FP32) != cudaSuccess) return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<FSE_PREC_FP32, false>, kThreads,
                                                      smem_bytes(iters)) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_block_loss(const FrameDesc *frames_dev, int n_frames, int max_rows_x_bw,
                              uint8_t *lost_out, uint8_t *part_out, const int *lost_off_dev,
                              cudaStream_t stream) {
    if (n_frames <= 0 || max_rows_x_bw <= 0) return cudaSuccess;
    dim3 grid((max_rows_x_bw + 255) / 256, n_frames);
    k_block_loss<<<grid, 256, 0, stream>>>(frames_dev, lost_out, part_out, lost_off_dev);
    return cudaGetLastError();
}

cudaError_t launch_wtables(const int32_t *keys, const uint64_t *dst, int n, float delta,
                           const float *rho_tab, const float2 *tw_tab, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = ensure_attrs(FSE_PREC_FP32);
    if (e != cudaSuccess) return e;
    k_wtable<<<n, kThreads, smem_bytes(0), stream>>>(keys, dst, delta, rho_tab, tw_tab);
    return cudaGetLastError();
}

cudaError_t launch_group(const FrameDesc *frames_dev, const int2 *items, int n_items,
                         const KParams &kp, const float *rho_tab, const float2 *tw_tab,
                         int precision, cudaStream_t stream) {
    if (!precision_supported(precision)) return cudaErrorInvalidValue;
    if (precision != FSE_PREC_FP32 && !kp.frags) return cudaErrorInvalidValue;
    cudaError_t e = ensure_attrs(precision);
    if (e != cudaSuccess) return e;
    if (n_items <= 0) return cudaSuccess;
    return with_precision(precision, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        k_group<P><<<n_items, kThreads, smem_bytes(kp.iters), stream>>>(frames_dev, items, kp,
                                                                        rho_tab, tw_tab);
        return cudaGetLastError();
    });
}

cudaError_t launch_persistent(const FrameDesc *frames_dev, const WorkQueue &wq,
                              const KParams &kp, const float *rho_tab, const float2 *tw_tab,
                              int precision, int grid, cudaStream_t stream) {
    if (!precision_supported(precision)) return cudaErrorInvalidValue;
    if (precision != FSE_PREC_FP32 && !kp.frags) return cudaErrorInvalidValue;
    cudaError_t e = ensure_attrs(precision);
    if (e != cudaSuccess) return e;
    if (wq.n <= 0) return cudaSuccess;
    if (kp.clocks) {  // phase stamps: FP32 projections only
        if (precision != FSE_PREC_FP32) return cudaErrorInvalidValue;
        k_persistent<FSE_PREC_FP32, true><<<grid, kThreads, smem_bytes(kp.iters), stream>>>(
            frames_dev, wq, kp, rho_tab, tw_tab);
        return cudaGetLastError();
    }
    return with_precision(precision, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        k_persistent<P, false><<<grid, kThreads, smem_bytes(kp.iters), stream>>>(
            frames_dev, wq, kp, rho_tab, tw_tab);
        return cudaGetLastError();
    });
}

cudaError_t launch_areas(const float *area_f, const uint8_t *area_cls, int n,
                         const KParams &kp, const float *rho_tab, const float2 *tw_tab,
                         int precision, float *g_out, int32_t *u_out, float *dc_out,
                         float *r_out, cudaStream_t stream) {
    if (!precision_supported(precision)) return cudaErrorInvalidValue;
    if (precision != FSE_PREC_FP32 && !kp.frags) return cudaErrorInvalidValue;
    cudaError_t e = ensure_attrs(precision);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    return with_precision(precision, [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        k_areas<P><<<n, kThreads, smem_bytes(kp.iters), stream>>>(
            area_f, area_cls, kp, rho_tab, tw_tab, g_out, u_out, dc_out, r_out);
        return cudaGetLastError();
    });
}

}  // namespace fse
