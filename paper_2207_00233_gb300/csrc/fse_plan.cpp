// Processing order of the blocks of one frame: the conventional line scan
// (Sec. 2) and the optimized, parallelizable order of Algorithm 1 (Sec. 3).
//
// Integer-only host code.  The counts N live in a grid padded by one block
// on every side so that the 8-neighbourhood needs no bounds tests; padding
// cells hold a sentinel that is never selected and never decremented.
//
// One implementation (plan_order_core) serves fse_plan_order, the frame
// paths and fse_conceal_frame_noalloc; it works in caller-provided scratch
// and allocates nothing.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/fse.h"
#include "fse_internal.h"

namespace {

constexpr int kPad = -0x40000000;  // padding cells: below every valid count
constexpr int kBuckets = 14;       // counts run from 0 to 8 neighbours + 5

inline int rim_penalty(int by, int bx, int bh, int bw) {
    const bool top_or_bottom = by == 0 || by == bh - 1;
    const bool left_or_right = bx == 0 || bx == bw - 1;
    if (top_or_bottom && left_or_right) return 5;  // corner block
    if (top_or_bottom || left_or_right) return 3;  // margin block
    return 0;
}

}  // namespace

namespace fse {

static_assert(kBuckets == 14, "plan_scratch_bytes assumes 14 candidate lists");

int plan_order_core(int bw, int bh, const uint8_t *block_lost, int order,
                    int32_t *group_of_block, int32_t *group_ptr, int32_t *block_ids,
                    int32_t *n_groups, void *scratch) {
    if (bw <= 0 || bh <= 0 || !block_lost || !group_of_block || !group_ptr || !block_ids ||
        !n_groups)
        return FSE_EINVAL;
    if (order != FSE_ORDER_LINESCAN && order != FSE_ORDER_OPTIMIZED) return FSE_EINVAL;
    if ((long long)bw * bh > (1LL << 28)) return FSE_EINVAL;
    const int nb = bw * bh;

    if (order == FSE_ORDER_LINESCAN) {
        int32_t g = 0;
        group_ptr[0] = 0;
        for (int b = 0; b < nb; ++b) {
            if (block_lost[b]) {
                block_ids[g] = b;
                group_of_block[b] = g++;
                group_ptr[g] = g;
            } else {
                group_of_block[b] = -1;
            }
        }
        *n_groups = g;
        return FSE_OK;
    }
    if (!scratch) return FSE_EINVAL;

    // Scratch: padded counts, candidate lists per count (each at most nb
    // entries: counts only decrease, so a block enters each list once), the
    // list lengths, and the padded membership of the set S being built.
    const int pw = bw + 2;
    const size_t padded = (size_t)pw * (bh + 2);
    int32_t *N = static_cast<int32_t *>(scratch);
    int32_t *bucket = N + padded;
    int32_t *blen = bucket + (size_t)kBuckets * nb;
    uint8_t *in_s = reinterpret_cast<uint8_t *>(blen + kBuckets);
    auto at = [&](int by, int bx) -> int32_t & { return N[(size_t)(by + 1) * pw + (bx + 1)]; };
    auto s_at = [&](int by, int bx) -> uint8_t & {
        return in_s[(size_t)(by + 1) * pw + (bx + 1)];
    };
    for (size_t i = 0; i < padded; ++i) N[i] = kPad;
    std::memset(in_s, 0, padded);
    for (int c = 0; c < kBuckets; ++c) blen[c] = 0;
    auto push = [&](int c, int b) { bucket[(size_t)c * nb + blen[c]++] = b; };

    // Initialisation pass of Algorithm 1: rim penalty for every block, and
    // +1 on each in-frame 8-neighbour of every lost block.
    for (int by = 0; by < bh; ++by)
        for (int bx = 0; bx < bw; ++bx) at(by, bx) = rim_penalty(by, bx, bh, bw);
    for (int by = 0; by < bh; ++by)
        for (int bx = 0; bx < bw; ++bx) {
            if (!block_lost[by * bw + bx]) continue;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    if (dy | dx) at(by + dy, bx + dx) += 1;  // padding stays very negative
        }
    // Second pass: blocks with nothing to extrapolate are marked -1.  The
    // others go into candidate lists by their count; entries whose count has
    // moved on are dropped lazily when their list is used.
    int pending = 0;
    for (int by = 0; by < bh; ++by)
        for (int bx = 0; bx < bw; ++bx) {
            const int b = by * bw + bx;
            if (!block_lost[b]) {
                at(by, bx) = -1;
                group_of_block[b] = -1;
                continue;
            }
            push(at(by, bx), b);
            ++pending;
        }

    int32_t g = 0, pos = 0;
    group_ptr[0] = 0;
    while (pending > 0) {
        // N_min: the smallest count with a live entry.  The live entries of
        // that list, in raster order, are exactly the blocks with N = N_min.
        int nmin = 0;
        for (;; ++nmin) {
            int32_t *lst = bucket + (size_t)nmin * nb;
            int k = 0;
            for (int i = 0; i < blen[nmin]; ++i)
                if (at(lst[i] / bw, lst[i] % bw) == nmin) lst[k++] = lst[i];
            blen[nmin] = k;
            if (k) break;
        }
        int32_t *cand = bucket + (size_t)nmin * nb;
        std::sort(cand, cand + blen[nmin]);
        // S: raster scan; a block joins when none of its neighbours joined
        // before it.  Only the left and the three upper neighbours can have
        // joined earlier in the scan.  Members go straight to block_ids.
        const int first = pos;
        for (int i = 0; i < blen[nmin]; ++i) {
            const int b = cand[i], by = b / bw, bx = b % bw;
            if (s_at(by, bx - 1) | s_at(by - 1, bx - 1) | s_at(by - 1, bx) |
                s_at(by - 1, bx + 1))
                continue;
            s_at(by, bx) = 1;
            block_ids[pos++] = b;
        }
        // Extrapolation of S, then the count updates of Algorithm 1.
        for (int i = first; i < pos; ++i) {
            const int b = block_ids[i], by = b / bw, bx = b % bw;
            group_of_block[b] = g;
            at(by, bx) = -1;
            s_at(by, bx) = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!(dy | dx)) continue;
                    // Only blocks still to do are decremented; finished
                    // blocks (-1) and padding keep their value.
                    int32_t &v = at(by + dy, bx + dx);
                    if (v >= 0) {
                        --v;
                        push(v, (by + dy) * bw + (bx + dx));
                    }
                }
        }
        pending -= pos - first;
        group_ptr[++g] = pos;
    }
    *n_groups = g;
    return FSE_OK;
}

}  // namespace fse

extern "C" int fse_plan_order(int bw, int bh, const uint8_t *block_lost,
                              int order, int32_t *group_of_block,
                              int32_t *group_ptr, int32_t *block_ids,
                              int32_t *n_groups) {
    if (bw <= 0 || bh <= 0 || (long long)bw * bh > (1LL << 28)) return FSE_EINVAL;
    std::vector<int32_t> scratch;
    if (order == FSE_ORDER_OPTIMIZED) {
        try {
            scratch.resize((fse::plan_scratch_bytes(bw, bh) + 3) / 4);
        } catch (...) {
            return FSE_ENOMEM;
        }
    }
    return fse::plan_order_core(bw, bh, block_lost, order, group_of_block, group_ptr,
                                block_ids, n_groups, scratch.empty() ? nullptr : scratch.data());
}
