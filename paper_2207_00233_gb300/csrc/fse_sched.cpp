// Claim order of the lost blocks of a batch for the device executors.
//
// Block s depends on block d when d is lost, lies within the area footprint
// of s (+-16/B blocks: the (B + 32)^2 area reaches that far) and belongs to
// an earlier group of the processing order (Sec. 3): s reads the concealed
// samples of d as class R.  Samples of blocks of the same or a later group
// are B_i / B_o for s, weigh 0 and are not read.  So any order in which every
// block comes after its dependencies gives the result of the group order.
//
// * Level order, for one launch per level: level(s) = 1 + the largest level
//   of its dependencies (0 without); blocks of one level are independent.
//   Levels are far fewer than groups (many groups do not touch each other).
// * Height order, for the persistent executor (P resident CTAs claim blocks
//   in order and wait for the dependencies of what they claimed): longest
//   chain of dependants first (the height of a block exceeds that of every
//   dependant, so the order is topological).  Long chains start early and
//   do not form a tail; a claim rarely waits.  Static: a counting sort.
// * Delayed height order, for the persistent executor: the height order cut
//   into rounds of P claims, each block moved to no earlier than the round
//   after its latest dependency's (dependencies first, per frame), then
//   sorted by round (within a round by frame, then group order).  A block
//   then rarely waits for a dependency claimed just before it; close to the
//   list schedule below, at the cost of one footprint scan per block, and
//   every pass runs per frame (in parallel) but for prefix sums.
// * Schedule (for comparison): list scheduling of P workers with unit
//   block times, longest chain first among the blocks whose dependencies
//   have started (ties: first ready first).  It waits even less, but costs
//   a footprint scan per block on the host; on the 16-frame 1080p batch it
//   saved 0.47 ms of a 17.9 ms kernel for 1.6 ms more host time than the
//   height order.

//
// Host code, integers only.
#include <algorithm>
#include <cstdint>
#include <functional>
#include <vector>

#include "../../include/fse.h"
#include "fse_internal.h"

namespace fse {

void frame_depths(FrameDepths &f, int rad) {
    f.rad = rad;
    f.pw = f.bw + 2 * rad;
    const int ph = f.bh + 2 * rad;
    f.gp.assign((size_t)f.pw * ph, -1);
    for (int y = 0; y < f.bh; ++y)
        std::copy(f.gob + (size_t)y * f.bw, f.gob + (size_t)(y + 1) * f.bw,
                  f.gp.begin() + (size_t)(y + rad) * f.pw + rad);
    f.nbr.clear();
    for (int dy = -rad; dy <= rad; ++dy)
        for (int dx = -rad; dx <= rad; ++dx)
            if (dy || dx) f.nbr.push_back(dy * f.pw + dx);
    f.level.assign(f.gp.size(), 0);
    f.height.assign(f.gp.size(), 0);
    f.indeg.assign(f.gp.size(), 0);
    f.pid.resize(f.n);
    const int32_t *gp = f.gp.data();
    for (int j = 0; j < f.n; ++j) {  // increasing group: dependencies first
        const int b = f.ids[j], by = b / f.bw, bx = b - by * f.bw;
        const int p = (by + rad) * f.pw + bx + rad;
        const uint32_t g = (uint32_t)gp[p];
        int lv = 0, deg = 0;
        for (const int32_t o : f.nbr) {  // branch-free: the tests are unpredictable
            const int dep = (uint32_t)gp[p + o] < g;  // 0 <= group < g (-1 wraps high)
            lv = std::max(lv, dep * (f.level[p + o] + 1));
            deg += dep;
        }
        f.pid[j] = p;
        f.level[p] = lv;
        f.indeg[p] = deg;
    }
    for (int j = f.n - 1; j >= 0; --j) {  // decreasing group: dependants first
        const int p = f.pid[j], g = gp[p];
        int h = 1;
        for (const int32_t o : f.nbr)
            h = std::max(h, (gp[p + o] > g) * (f.height[p + o] + 1));
        f.height[p] = h;
    }
}

void level_claims(const std::vector<FrameDepths> &frames, std::vector<int2> &items,
                  std::vector<int> &level_start) {
    int n_levels = 0;
    size_t total = 0;
    for (const FrameDepths &f : frames) {
        total += f.n;
        for (int j = 0; j < f.n; ++j) n_levels = std::max(n_levels, f.level[f.pid[j]] + 1);
    }
    // counting sort by level; within a level by frame, then group order
    level_start.assign(n_levels + 1, 0);
    for (const FrameDepths &f : frames)
        for (int j = 0; j < f.n; ++j) ++level_start[f.level[f.pid[j]] + 1];
    for (int l = 0; l < n_levels; ++l) level_start[l + 1] += level_start[l];
    std::vector<int> fill(level_start.begin(), level_start.end() - 1);
    items.assign(total, make_int2(0, 0));
    for (size_t i = 0; i < frames.size(); ++i) {
        const FrameDepths &f = frames[i];
        for (int j = 0; j < f.n; ++j)
            items[fill[f.level[f.pid[j]]]++] = make_int2((int)i, f.ids[j]);
    }
}

namespace {

// (frame, position in the frame's group order) of every lost block, longest
// chain of dependants first; within a height by frame, then group order.
void height_order(const std::vector<FrameDepths> &frames, std::vector<int2> &order) {
    int max_h = 0;
    size_t total = 0;
    for (const FrameDepths &f : frames) {
        total += f.n;
        for (int j = 0; j < f.n; ++j) max_h = std::max(max_h, f.height[f.pid[j]]);
    }
    std::vector<size_t> start(max_h + 2, 0);
    for (const FrameDepths &f : frames)
        for (int j = 0; j < f.n; ++j) ++start[max_h - f.height[f.pid[j]] + 1];
    for (int h = 0; h <= max_h; ++h) start[h + 1] += start[h];
    order.assign(total, make_int2(0, 0));
    for (size_t i = 0; i < frames.size(); ++i) {
        const FrameDepths &f = frames[i];
        for (int j = 0; j < f.n; ++j) order[start[max_h - f.height[f.pid[j]]]++] = make_int2((int)i, j);
    }
}

}  // namespace

void height_claims(const std::vector<FrameDepths> &frames, std::vector<int2> &items) {
    height_order(frames, items);
    for (int2 &it : items) it.y = frames[it.x].ids[it.y];
}

void delay_claims(std::vector<FrameDepths> &frames, int workers, std::vector<int2> &items,
                  const std::function<void(int, const std::function<void(int)> &)> &pfor) {
    const int nf = (int)frames.size();
    const size_t P = (size_t)std::max(workers, 1);
    // Per-frame histograms by height; every step below is per frame except
    // for prefix sums over (height or round, frame).
    int max_h = 0;
    for (const FrameDepths &f : frames)
        for (int j = 0; j < f.n; ++j) max_h = std::max(max_h, f.height[f.pid[j]]);
    std::vector<std::vector<int32_t>> hist(nf);
    pfor(nf, [&](int i) {
        FrameDepths &f = frames[i];
        hist[i].assign(max_h + 1, 0);
        for (int j = 0; j < f.n; ++j) ++hist[i][f.height[f.pid[j]]];
    });
    // rank of the first block of (height, frame) in the height order
    // (height descending, then frame, then group order)
    std::vector<std::vector<size_t>> first(nf, std::vector<size_t>(max_h + 1));
    size_t pos = 0;
    for (int h = max_h; h >= 1; --h)
        for (int i = 0; i < nf; ++i) {
            first[i][h] = pos;
            pos += hist[i][h];
        }
    // round of each block in the height order, then no earlier than the
    // round after the latest dependency's (dependencies first: group order)
    std::vector<int32_t> max_key(nf, 0);
    pfor(nf, [&](int i) {
        FrameDepths &f = frames[i];
        f.key.assign(f.gp.size(), 0);
        std::vector<size_t> next(first[i]);
        const int32_t *gp = f.gp.data();
        int32_t mk = 0;
        for (int j = 0; j < f.n; ++j) {
            const int p = f.pid[j];
            const uint32_t g = (uint32_t)gp[p];
            int k = (int)(next[f.height[p]]++ / P);
            for (const int32_t o : f.nbr)
                if ((uint32_t)gp[p + o] < g) k = std::max(k, f.key[p + o] + 1);
            f.key[p] = k;
            mk = std::max(mk, k);
        }
        max_key[i] = mk;
    });
    // items by round; within a round by frame, then group order
    int mk = 0;
    for (int i = 0; i < nf; ++i) mk = std::max(mk, max_key[i]);
    pfor(nf, [&](int i) {
        const FrameDepths &f = frames[i];
        hist[i].assign(mk + 1, 0);
        for (int j = 0; j < f.n; ++j) ++hist[i][f.key[f.pid[j]]];
    });
    pos = 0;
    for (int k = 0; k <= mk; ++k)
        for (int i = 0; i < nf; ++i) {
            const int32_t c = hist[i][k];
            hist[i][k] = (int32_t)pos;  // now the first slot of (round, frame)
            pos += c;
        }
    items.assign(pos, make_int2(0, 0));
    pfor(nf, [&](int i) {
        const FrameDepths &f = frames[i];
        for (int j = 0; j < f.n; ++j) items[hist[i][f.key[f.pid[j]]]++] = make_int2(i, f.ids[j]);
    });
}

void schedule_claims(std::vector<FrameDepths> &frames, int workers, std::vector<int2> &items) {
    // Ready blocks in buckets by height (the longest chain first); a bucket
    // is a FIFO of (frame, padded cell): initially frame by frame in group
    // order, then in the order of release.  Heights are at most the number
    // of groups of a frame.
    int max_h = 0;
    size_t total = 0;
    for (const FrameDepths &f : frames) {
        total += f.n;
        for (int j = 0; j < f.n; ++j) max_h = std::max(max_h, f.height[f.pid[j]]);
    }
    std::vector<std::vector<int2>> bucket(max_h + 1);
    std::vector<size_t> head(max_h + 1, 0);
    for (size_t i = 0; i < frames.size(); ++i) {
        const FrameDepths &f = frames[i];
        for (int j = 0; j < f.n; ++j) {
            const int p = f.pid[j];
            if (f.indeg[p] == 0) bucket[f.height[p]].push_back(make_int2((int)i, p));
        }
    }
    items.clear();
    items.reserve(total);
    const size_t P = (size_t)std::max(workers, 1);
    std::vector<int2> released;
    int top = max_h;  // no ready block is higher
    while (items.size() < total) {
        released.clear();
        for (size_t t = 0; t < P; ++t) {
            while (top > 0 && head[top] == bucket[top].size()) --top;
            if (head[top] == bucket[top].size()) break;  // nothing ready
            const int2 it = bucket[top][head[top]++];
            FrameDepths &f = frames[it.x];
            items.push_back(make_int2(it.x, f.block_of(it.y)));
            const int g = f.gp[it.y];
            for (const int32_t o : f.nbr) {
                const int q = it.y + o;
                const int dep = f.gp[q] > g;  // q waits for this block
                f.indeg[q] -= dep;
                if (dep & (f.indeg[q] == 0)) released.push_back(make_int2(it.x, q));
            }
        }
        if (released.empty() && head[top] == bucket[top].size())
            break;  // nothing left to start (all blocks were, for a consistent plan)
        for (const int2 &r : released) {
            const int h = frames[r.x].height[r.y];
            bucket[h].push_back(r);
            top = std::max(top, h);
        }
    }
}

}  // namespace fse

extern "C" int fse_plan_claims(int n_frames, const int32_t *bw, const int32_t *bh,
                               const int32_t *group_of_block, int block, int workers, int mode,
                               int32_t *items, int32_t *level_start, int32_t *n_levels) {
    using namespace fse;
    const int lb = block_log2(block);
    if (n_frames <= 0 || !bw || !bh || !group_of_block || !items || lb < 0 || mode < 0 ||
        mode > 3 || (mode == 0 && (!level_start || !n_levels)) ||
        ((mode == 1 || mode == 3) && workers <= 0))
        return FSE_EINVAL;
    std::vector<FrameDepths> frames(n_frames);
    size_t off = 0;
    for (int i = 0; i < n_frames; ++i) {
        if (bw[i] <= 0 || bh[i] <= 0) return FSE_EINVAL;
        FrameDepths &f = frames[i];
        f.bw = bw[i];
        f.bh = bh[i];
        f.gob = group_of_block + off;
        off += (size_t)bw[i] * bh[i];
        // lost blocks in group order (ties: raster order)
        std::vector<int32_t> ids;
        for (int b = 0; b < f.bw * f.bh; ++b)
            if (f.gob[b] >= 0) ids.push_back(b);
        std::stable_sort(ids.begin(), ids.end(),
                         [&](int32_t a, int32_t c) { return f.gob[a] < f.gob[c]; });
        f.own_ids = std::move(ids);
        f.ids = f.own_ids.data();
        f.n = (int)f.own_ids.size();
        frame_depths(f, kBorder >> lb);
    }
    std::vector<int2> out;
    if (mode == 0) {
        std::vector<int> ls;
        level_claims(frames, out, ls);
        *n_levels = (int32_t)ls.size() - 1;
        for (size_t l = 0; l < ls.size(); ++l) level_start[l] = ls[l];
    } else if (mode == 1) {
        schedule_claims(frames, workers, out);
    } else {
        if (mode == 2)
            height_claims(frames, out);
        else
            delay_claims(frames, workers, out, [](int n, const std::function<void(int)> &fn) {
                for (int i = 0; i < n; ++i) fn(i);
            });
    }
    for (size_t k = 0; k < out.size(); ++k) {
        items[2 * k] = out[k].x;
        items[2 * k + 1] = out[k].y;
    }
    return FSE_OK;
}
