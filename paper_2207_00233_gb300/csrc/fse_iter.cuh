// Building blocks of the FSE iteration loop (Sec. 4: per iteration, select
// u = argmax_k |R_w[k]|^2, ties to the smallest linear index 64 k_m + k_n;
// dc = gamma R_w[u] / W[0]; R_w[k] -= dc W[(k - u) mod 64] for all k).
//
// Shared by the per-block kernels (fse_kernels.cu) and the loop
// microbenchmark (fse_loopbench.cu), so that the microbenchmark times the
// product's loop body.
//
// Register layout: thread (warp w, lane l) of a 256-thread CTA owns the 16
// spectrum entries k_m = 8w + r (r = 0..7), k_n in {l, l + 32}; each row r
// is held as two packed f32x2 registers (real parts, imaginary parts).
// W lives in shared memory in the W4 layout of fse_internal.h: one 16-byte
// load gives a thread W at both of its columns.
#pragma once

#include <cstdint>

#include "fse_internal.h"

namespace fse {
namespace iter {

typedef unsigned long long u64;

// ---- packed FP32 pairs ------------------------------------------------------
__device__ __forceinline__ u64 pack2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpack2(u64 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// |R|^2 of a pair; the same instruction sequence is used wherever an
// energy is compared, so equal inputs give bit-identical energies.
__device__ __forceinline__ u64 energy2(u64 re, u64 im) {
    return fma2(im, im, mul2(re, re));
}
__device__ __forceinline__ float max3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ void lds_pair(uint32_t addr, u64 &a, u64 &b) {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void st_shared_pair(uint32_t addr, u64 a, u64 b) {
    asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

// Shared address of W4[(8w - u_m) mod 64][(l - u_n) mod 64] for this thread.
__device__ __forceinline__ uint32_t w4_base(uint32_t w4addr, int um, int un) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int row = (8 * w - um) & (kDft - 1);
    const int col = (l - un) & (kDft - 1);
    return w4addr + (uint32_t)(row * kDft + col) * 16u;
}

// One row of the update: R -= dc * W[k - u] for the thread's two entries of
// row r (dc = 0 leaves R bit-identical); returns their energies.
__device__ __forceinline__ float2 update_row(uint32_t wbase, int r, u64 ndcr2, u64 dci2,
                                             u64 ndci2, u64 &rre, u64 &rim) {
    u64 wr, wi;
    lds_pair(wbase + r * (kDft * 16), wr, wi);
    u64 a = fma2(wr, ndcr2, rre);
    a = fma2(wi, dci2, a);
    u64 b = fma2(wi, ndcr2, rim);
    b = fma2(wr, ndci2, b);
    rre = a;
    rim = b;
    return unpack2(energy2(a, b));
}

// ---- selection: two block barriers -------------------------------------------
//
// Warp maxima -> barrier -> block maximum; the warps that hold it search
// their entries for the smallest index -> barrier -> the smallest candidate.
// smax: [8] words, cand: [8] float4 (index bits, Re, Im, -).
__device__ __forceinline__ float update_and_max(uint32_t wbase, u64 ndcr2, u64 dci2,
                                                u64 ndci2, u64 (&rre)[8], u64 (&rim)[8]) {
    float mx = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 e = update_row(wbase, r, ndcr2, dci2, ndci2, rre[r], rim[r]);
        mx = max3(mx, e.x, e.y);
    }
    return mx;
}

__device__ __forceinline__ void select_two_barriers(float tmx, const u64 (&rre)[8],
                                                    const u64 (&rim)[8], uint32_t *smax,
                                                    float4 *cand, uint32_t &u, float &ure,
                                                    float &uim) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(tmx));
    if (l == 0) smax[w] = wmx;
    __syncthreads();
    // lanes 0..7 read the eight warp maxima in one access
    const uint32_t estar = __reduce_max_sync(0xffffffffu, l < kWarps ? smax[l] : 0u);
    // Smallest linear index whose energy equals the maximum.  Only the warps
    // that hold the maximum search (a warp-uniform branch).
    if (__any_sync(0xffffffffu, __float_as_uint(tmx) == estar)) {
        uint32_t kk = 0xffffffffu;
        float cre = 0.f, cim = 0.f;
        if (__float_as_uint(tmx) == estar) {
#pragma unroll
            for (int r = 7; r >= 0; --r) {
                const float2 e = unpack2(energy2(rre[r], rim[r]));
                const float2 re = unpack2(rre[r]), im = unpack2(rim[r]);
                if (__float_as_uint(e.y) == estar) {
                    kk = (uint32_t)((8 * w + r) * kDft + l + 32);
                    cre = re.y;
                    cim = im.y;
                }
                if (__float_as_uint(e.x) == estar) {
                    kk = (uint32_t)((8 * w + r) * kDft + l);
                    cre = re.x;
                    cim = im.x;
                }
            }
        }
        // the lane holding the warp's smallest index writes its candidate
        const uint32_t wk = __reduce_min_sync(0xffffffffu, kk);
        if (kk == wk) cand[w] = make_float4(__uint_as_float(wk), cre, cim, 0.f);
    } else if (l == 0) {
        cand[w].x = __uint_as_float(0xffffffffu);
    }
    __syncthreads();
    // lanes 0..7 read the eight warp candidates; the smallest index wins.
    // Warp w owns indices [512 w, 512 w + 512), so the winner's slot is u >> 9.
    u = __reduce_min_sync(0xffffffffu,
                          l < kWarps ? __float_as_uint(cand[l].x) : 0xffffffffu);
    const float4 cw = cand[(u >> 9) & (kWarps - 1)];
    ure = cw.y;
    uim = cw.z;
}

// ---- selection: two block barriers, fewer shared-memory round trips ----------
//
// The same selection as select_two_barriers with two of its dependent
// shared-memory accesses replaced.  kAtomic: each warp's maximum goes into a
// single word with a shared atomic maximum, so after the first barrier a
// broadcast load gives the block maximum without a second reduction (two
// words alternate by iteration parity: thread 0 clears the one the next
// iteration uses, whose last reads came before this iteration's first
// barrier; both start at zero).  In every form the eight candidates are read
// once after the second barrier (lane l reads slot l mod 8) and the winner's
// value comes from its lane by shuffles instead of a dependent load.
template <bool kAtomic>
__device__ __forceinline__ void select_two_barriers_v2(float tmx, const u64 (&rre)[8],
                                                       const u64 (&rim)[8], uint32_t *smax,
                                                       float4 *cand, int it, uint32_t &u,
                                                       float &ure, float &uim) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(tmx));
    uint32_t estar;
    if (kAtomic) {
        if (l == 0) atomicMax(smax + (it & 1), wmx);
        __syncthreads();
        estar = smax[it & 1];
        if (threadIdx.x == 0) smax[(it + 1) & 1] = 0u;
    } else {
        if (l == 0) smax[w] = wmx;
        __syncthreads();
        estar = __reduce_max_sync(0xffffffffu, smax[l & (kWarps - 1)]);
    }
    if (__any_sync(0xffffffffu, __float_as_uint(tmx) == estar)) {
        uint32_t kk = 0xffffffffu;
        float cre = 0.f, cim = 0.f;
        if (__float_as_uint(tmx) == estar) {
#pragma unroll
            for (int r = 7; r >= 0; --r) {
                const float2 e = unpack2(energy2(rre[r], rim[r]));
                const float2 re = unpack2(rre[r]), im = unpack2(rim[r]);
                if (__float_as_uint(e.y) == estar) {
                    kk = (uint32_t)((8 * w + r) * kDft + l + 32);
                    cre = re.y;
                    cim = im.y;
                }
                if (__float_as_uint(e.x) == estar) {
                    kk = (uint32_t)((8 * w + r) * kDft + l);
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
    const float4 c = cand[l & (kWarps - 1)];
    u = __reduce_min_sync(0xffffffffu, __float_as_uint(c.x));
    // warp w owns the indices [512 w, 512 w + 512): the winner's slot, and
    // the lane that read it, is u >> 9
    const int ws = (int)((u >> 9) & (kWarps - 1));
    ure = __shfl_sync(0xffffffffu, c.y, ws);
    uim = __shfl_sync(0xffffffffu, c.z, ws);
}

// ---- selection: two block barriers, the winning warp named by its maximum -----
//
// Warp maxima -> barrier -> every warp reads the eight maxima and names the
// winning warp: the smallest warp holding the block maximum (warp w owns the
// indices [512 w, 512 w + 512), so the smallest index lies there).  Only
// that warp searches; its lane with the smallest index computes
// dc = gamma R_w[u] / W[0], writes the coefficient list entry and publishes
// everything the update needs, pre-packed, in one 32-byte slot:
// (-dc_r, -dc_r, dc_i, dc_i), (-dc_i, -dc_i, u_m << 10, u_n << 4) -> barrier
// -> every thread loads the slot.
struct Step {
    u64 ndcr2, dci2, ndci2;  // packed update constants
    uint32_t rowoff, coloff; // u_m * 1024, u_n * 16 (W4 byte offsets)
};

// The thread's smallest slot s (= 2 r for column l, 2 r + 1 for l + 32) whose
// energy equals estar, found with a match mask and a selection tree; kk is
// its linear index (all ones if no slot matches).
__device__ __forceinline__ void search_tree(uint32_t estar, const u64 (&rre)[8],
                                            const u64 (&rim)[8], uint32_t &kk, float &cre,
                                            float &cim) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint32_t m[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 e = unpack2(energy2(rre[r], rim[r]));
        m[r] = (__float_as_uint(e.x) == estar ? 1u : 0u) | (__float_as_uint(e.y) == estar ? 2u : 0u);
    }
    const uint32_t mask = ((m[0] | (m[1] << 2)) | ((m[2] << 4) | (m[3] << 6))) |
                          (((m[4] << 8) | (m[5] << 10)) | ((m[6] << 12) | (m[7] << 14)));
    const int sl = __ffs(mask) - 1;
    const bool b1 = (sl >> 1) & 1, b2 = (sl >> 2) & 1, b3 = (sl >> 3) & 1;
    const u64 a0 = b1 ? rre[1] : rre[0], a1 = b1 ? rre[3] : rre[2];
    const u64 a2 = b1 ? rre[5] : rre[4], a3 = b1 ? rre[7] : rre[6];
    const u64 c0 = b1 ? rim[1] : rim[0], c1 = b1 ? rim[3] : rim[2];
    const u64 c2 = b1 ? rim[5] : rim[4], c3 = b1 ? rim[7] : rim[6];
    const u64 ar = b3 ? (b2 ? a3 : a2) : (b2 ? a1 : a0);
    const u64 ci = b3 ? (b2 ? c3 : c2) : (b2 ? c1 : c0);
    const float2 re = unpack2(ar), im = unpack2(ci);
    const bool hi = sl & 1;
    cre = hi ? re.y : re.x;
    cim = hi ? im.y : im.x;
    kk = mask ? (uint32_t)((8 * w + (sl >> 1)) * kDft + l + (hi ? 32 : 0)) : 0xffffffffu;
}

// The winning lane's stores: the coefficient list entry (dc, u) and the
// update step (-dc_r, -dc_r, dc_i, dc_i), (-dc_i, -dc_i, u_m << 10, u_n << 4).
// Written as predicated stores rather than a branch on the lane: a
// single-lane branch in the loop made the block kernel 2.8% slower.
__device__ __forceinline__ void publish_step(bool win, float2 *dcl_it, uint16_t *ul_it,
                                             uint4 *slot, float dcr, float dci, uint32_t wk) {
    asm volatile(
        "{ .reg .pred q; setp.ne.u32 q, %0, 0;\n"
        "@q st.shared.v2.f32 [%1], {%2, %3};\n"
        "@q st.shared.u16 [%4], %5;\n"
        "@q st.shared.v4.b32 [%6], {%7, %7, %8, %8};\n"
        "@q st.shared.v4.b32 [%6+16], {%9, %9, %10, %11}; }"
        ::"r"(win ? 1u : 0u), "r"(smem_addr(dcl_it)), "f"(dcr), "f"(dci), "r"(smem_addr(ul_it)),
        "h"((unsigned short)wk), "r"(smem_addr(slot)), "r"(__float_as_uint(-dcr)),
        "r"(__float_as_uint(dci)), "r"(__float_as_uint(-dci)), "r"((wk >> 6) << 10),
        "r"((wk & 63) << 4)
        : "memory");
}

template <bool kTree>
__device__ __forceinline__ void select_named_warp(float tmx, const u64 (&rre)[8],
                                                  const u64 (&rim)[8], float gw, int it,
                                                  uint32_t *smax, uint4 *slot, float2 *dcl,
                                                  uint16_t *ul, Step &st) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(tmx));
    smax[w] = wmx;  // every lane stores the same value: no single-lane branch (2% faster)
    __syncthreads();
    const uint32_t v = smax[l & (kWarps - 1)];
    const uint32_t estar = __reduce_max_sync(0xffffffffu, v);
    const int wstar = __ffs(__ballot_sync(0xffffffffu, v == estar) & ((1u << kWarps) - 1u)) - 1;
    // The winning warp's test as a warp vote: the compiler sees a value
    // uniform across the warp (w == wstar is too, but not visibly), and the
    // block kernel runs 1.5% faster.
    if (__any_sync(0xffffffffu, w == wstar)) {
        // Every lane of the winning warp searches (no branch on its own
        // maximum: a lane whose maximum is below estar matches no entry,
        // and the block kernel runs 3.7% faster without the divergence).
        uint32_t kk = 0xffffffffu;
        float cre = 0.f, cim = 0.f;
        {
            if (kTree) {
                search_tree(estar, rre, rim, kk, cre, cim);
            } else {
#pragma unroll
                for (int r = 7; r >= 0; --r) {
                    const float2 e = unpack2(energy2(rre[r], rim[r]));
                    const float2 re = unpack2(rre[r]), im = unpack2(rim[r]);
                    if (__float_as_uint(e.y) == estar) {
                        kk = (uint32_t)((8 * w + r) * kDft + l + 32);
                        cre = re.y;
                        cim = im.y;
                    }
                    if (__float_as_uint(e.x) == estar) {
                        kk = (uint32_t)((8 * w + r) * kDft + l);
                        cre = re.x;
                        cim = im.x;
                    }
                }
            }
        }
        const uint32_t wk = __reduce_min_sync(0xffffffffu, kk);
        const float dcr = cre * gw, dci = cim * gw;
        publish_step(kk == wk, dcl + it, ul + it, slot, dcr, dci, wk);
    }
    __syncthreads();
    u64 a0, a1, b0, b1;
    lds_pair(smem_addr(slot), a0, a1);
    lds_pair(smem_addr(slot + 1), b0, b1);
    st.ndcr2 = a0;
    st.dci2 = a1;
    st.ndci2 = b0;
    st.rowoff = (uint32_t)b1;
    st.coloff = (uint32_t)(b1 >> 32);
}

// Shared address of W4[(8w - u_m) mod 64][(l - u_n) mod 64] from the
// published offsets; w8k = 8w * 1024, l16 = 16 l.
__device__ __forceinline__ uint32_t w4_addr_of(uint32_t w4addr, uint32_t w8k, uint32_t l16,
                                               const Step &st) {
    return w4addr + ((w8k - st.rowoff) & 0xFC00u) + ((l16 - st.coloff) & 0x3F0u);
}

// ---- selection: one block barrier, row maxima reduced during the update ------
//
// Every row of the thread's entries is reduced over the warp as soon as it
// is updated (a warp-uniform value), so after the update the warp knows its
// maximum and the smallest row that holds it; in that row the smallest
// column with the maximum is found by two ballots.  Each warp publishes its
// candidate (energy, index, Re, Im) in one 16-byte slot, and after a single
// barrier every warp picks the largest energy, ties to the smallest warp
// (warp w owns the indices [512 w, 512 w + 512)).  Slots are double-buffered
// by iteration parity: the slots written in iteration it + 2 were last read
// before the barrier of iteration it + 1.
__device__ __forceinline__ void update_rowmax(uint32_t wbase, u64 ndcr2, u64 dci2, u64 ndci2,
                                              u64 (&rre)[8], u64 (&rim)[8], uint32_t &wm,
                                              int &rs) {
    wm = 0u;
    rs = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 e = update_row(wbase, r, ndcr2, dci2, ndci2, rre[r], rim[r]);
        const uint32_t v = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(e.x, e.y)));
        if (v > wm) {  // strictly larger: the smallest row keeps a tie
            wm = v;
            rs = r;
        }
    }
}

__device__ __forceinline__ void publish_row_candidate(uint32_t wm, int rs, const u64 (&rre)[8],
                                                      const u64 (&rim)[8], uint4 *slots) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    u64 sre = rre[0], sim = rim[0];
#pragma unroll
    for (int r = 1; r < 8; ++r)
        if (rs == r) {
            sre = rre[r];
            sim = rim[r];
        }
    const float2 e = unpack2(energy2(sre, sim));
    const uint32_t bx = __ballot_sync(0xffffffffu, __float_as_uint(e.x) == wm);
    const uint32_t by = __ballot_sync(0xffffffffu, __float_as_uint(e.y) == wm);
    const bool left = bx != 0u;  // columns l (0..31) precede columns l + 32
    const int src = __ffs(left ? bx : by) - 1;
    if (l == src) {
        const float2 re = unpack2(sre), im = unpack2(sim);
        slots[w] = make_uint4(wm, (uint32_t)((8 * w + rs) * kDft + l + (left ? 0 : 32)),
                              __float_as_uint(left ? re.x : re.y),
                              __float_as_uint(left ? im.x : im.y));
    }
}

// After the barrier: the block's selection from the eight published slots.
__device__ __forceinline__ void pick_candidate(const uint4 *slots, uint32_t &u, float &ure,
                                               float &uim) {
    const int l = threadIdx.x & 31;
    const uint4 c = slots[l & (kWarps - 1)];
    const uint32_t emax = __reduce_max_sync(0xffffffffu, c.x);
    const uint32_t hit = __ballot_sync(0xffffffffu, c.x == emax) & ((1u << kWarps) - 1u);
    const int ws = __ffs(hit) - 1;
    u = __shfl_sync(0xffffffffu, c.y, ws);
    ure = __uint_as_float(__shfl_sync(0xffffffffu, c.z, ws));
    uim = __uint_as_float(__shfl_sync(0xffffffffu, c.w, ws));
}

// ---- selection: one block barrier, every warp searches its own maximum -------
__device__ __forceinline__ void publish_searched_candidate(float tmx, const u64 (&rre)[8],
                                                          const u64 (&rim)[8], uint4 *slots) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t wmx = __reduce_max_sync(0xffffffffu, __float_as_uint(tmx));
    uint32_t kk = 0xffffffffu;
    float cre = 0.f, cim = 0.f;
    if (__float_as_uint(tmx) == wmx) {
#pragma unroll
        for (int r = 7; r >= 0; --r) {
            const float2 e = unpack2(energy2(rre[r], rim[r]));
            const float2 re = unpack2(rre[r]), im = unpack2(rim[r]);
            if (__float_as_uint(e.y) == wmx) {
                kk = (uint32_t)((8 * w + r) * kDft + l + 32);
                cre = re.y;
                cim = im.y;
            }
            if (__float_as_uint(e.x) == wmx) {
                kk = (uint32_t)((8 * w + r) * kDft + l);
                cre = re.x;
                cim = im.x;
            }
        }
    }
    const uint32_t wk = __reduce_min_sync(0xffffffffu, kk);
    if (kk == wk) slots[w] = make_uint4(wmx, wk, __float_as_uint(cre), __float_as_uint(cim));
}

}  // namespace iter
}  // namespace fse
