// Processing order of the blocks of one frame: the conventional line scan
// (Sec. 2) and the optimized, parallelizable order of Algorithm 1 (Sec. 3).
//
// Integer-only host code.  The counts N live in a grid padded by one block
// on every side so that the 8-neighbourhood needs no bounds tests; padding
// cells hold a sentinel that is never selected and never decremented.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/fse.h"

namespace {

constexpr int kPad = -0x40000000;  // padding cells: below every valid count

struct Grid {
    int bw, bh, pw;  // pw = bw + 2
    std::vector<int> n;
    int &at(int by, int bx) { return n[(size_t)(by + 1) * pw + (bx + 1)]; }
};

inline int rim_penalty(int by, int bx, int bh, int bw) {
    const bool top_or_bottom = by == 0 || by == bh - 1;
    const bool left_or_right = bx == 0 || bx == bw - 1;
    if (top_or_bottom && left_or_right) return 5;  // corner block
    if (top_or_bottom || left_or_right) return 3;  // margin block
    return 0;
}

}  // namespace

extern "C" int fse_plan_order(int bw, int bh, const uint8_t *block_lost,
                              int order, int32_t *group_of_block,
                              int32_t *group_ptr, int32_t *block_ids,
                              int32_t *n_groups) {
    if (bw <= 0 || bh <= 0 || !block_lost || !group_of_block || !group_ptr ||
        !block_ids || !n_groups)
        return FSE_EINVAL;
    if (order != FSE_ORDER_LINESCAN && order != FSE_ORDER_OPTIMIZED)
        return FSE_EINVAL;
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

    Grid G{bw, bh, bw + 2, std::vector<int>((size_t)(bw + 2) * (bh + 2), kPad)};
    // Initialisation pass of Algorithm 1: rim penalty for every block, and
    // +1 on each in-frame 8-neighbour of every lost block.
    for (int by = 0; by < bh; ++by)
        for (int bx = 0; bx < bw; ++bx) G.at(by, bx) = rim_penalty(by, bx, bh, bw);
    for (int by = 0; by < bh; ++by)
        for (int bx = 0; bx < bw; ++bx) {
            if (!block_lost[by * bw + bx]) continue;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                    if (dy | dx) G.at(by + dy, bx + dx) += 1;  // padding stays very negative
        }
    // Second pass: blocks with nothing to extrapolate are marked -1.  The
    // others go into candidate lists by their count.  Counts only decrease,
    // so a block is appended to each list at most once; entries whose count
    // has moved on are dropped lazily when their list is used.
    std::vector<std::vector<int>> bucket(16);
    int pending = 0;
    for (int by = 0; by < bh; ++by)
        for (int bx = 0; bx < bw; ++bx) {
            const int b = by * bw + bx;
            if (!block_lost[b]) {
                G.at(by, bx) = -1;
                group_of_block[b] = -1;
                continue;
            }
            bucket[G.at(by, bx)].push_back(b);  // counts are at most 8 + 5
            ++pending;
        }

    // Membership of the set S under construction, padded like G.
    std::vector<uint8_t> in_s((size_t)(bw + 2) * (bh + 2), 0);
    auto s_at = [&](int by, int bx) -> uint8_t & {
        return in_s[(size_t)(by + 1) * G.pw + (bx + 1)];
    };

    int32_t g = 0, pos = 0;
    group_ptr[0] = 0;
    std::vector<int> members;
    while (pending > 0) {
        // N_min: the smallest count with a live entry.  The live entries of
        // that list, in raster order, are exactly the blocks with N = N_min.
        int nmin = 0;
        for (;; ++nmin) {
            std::vector<int> &lst = bucket[nmin];
            size_t k = 0;
            for (int b : lst)
                if (G.at(b / bw, b % bw) == nmin) lst[k++] = b;
            lst.resize(k);
            if (k) break;
        }
        std::vector<int> &cand = bucket[nmin];
        std::sort(cand.begin(), cand.end());
        // S: raster scan; a block joins when none of its neighbours joined
        // before it.  Only the left and the three upper neighbours can have
        // joined earlier in the scan.
        members.clear();
        for (int b : cand) {
            const int by = b / bw, bx = b % bw;
            if (s_at(by, bx - 1) | s_at(by - 1, bx - 1) | s_at(by - 1, bx) |
                s_at(by - 1, bx + 1))
                continue;
            s_at(by, bx) = 1;
            members.push_back(b);
        }
        // Extrapolation of S, then the count updates of Algorithm 1.
        for (int b : members) {
            const int by = b / bw, bx = b % bw;
            block_ids[pos++] = b;
            group_of_block[b] = g;
            G.at(by, bx) = -1;
            s_at(by, bx) = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!(dy | dx)) continue;
                    // Only blocks still to do are decremented; finished
                    // blocks (-1) and padding keep their value.
                    int &v = G.at(by + dy, bx + dx);
                    if (v >= 0) {
                        --v;
                        bucket[v].push_back((by + dy) * bw + (bx + dx));
                    }
                }
        }
        pending -= (int)members.size();
        group_ptr[++g] = pos;
    }
    *n_groups = g;
    return FSE_OK;
}
