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
// * Schedule, for the persistent executor (P resident CTAs claim blocks in
//   order and wait for the dependencies of what they claimed): list
//   scheduling with unit block times, longest chain of dependants first.
//   Each round starts the P ready blocks whose chains to the end are
//   longest; dependants become ready in the next round.  Claims in that
//   order rarely wait, and long chains start early enough not to form a
//   tail.
//
// Host code, integers only.
#include <algorithm>
#include <cstdint>
#include <queue>
#include <vector>

#include "../../include/fse.h"
#include "fse_internal.h"

namespace fse {

void frame_depths(FrameDepths &f, int rad) {
    const int nb = f.bw * f.bh;
    f.level.assign(nb, -1);
    f.height.assign(nb, 0);
    f.indeg.assign(nb, 0);
    f.pos.assign(nb, -1);
    const int32_t *gob = f.gob;
    for (int j = 0; j < f.n; ++j) {  // increasing group
        const int b = f.ids[j], by = b / f.bw, bx = b - by * f.bw, g = gob[b];
        int lv = 0, deg = 0;
        for (int y = std::max(0, by - rad); y <= std::min(f.bh - 1, by + rad); ++y)
            for (int x = std::max(0, bx - rad); x <= std::min(f.bw - 1, bx + rad); ++x) {
                const int d = y * f.bw + x;
                if (gob[d] >= 0 && gob[d] < g) {
                    lv = std::max(lv, f.level[d] + 1);
                    ++deg;
                }
            }
        f.level[b] = lv;
        f.indeg[b] = deg;
        f.pos[b] = j;
    }
    for (int j = f.n - 1; j >= 0; --j) {  // decreasing group: dependants first
        const int b = f.ids[j], by = b / f.bw, bx = b - by * f.bw, g = gob[b];
        int h = 1;
        for (int y = std::max(0, by - rad); y <= std::min(f.bh - 1, by + rad); ++y)
            for (int x = std::max(0, bx - rad); x <= std::min(f.bw - 1, bx + rad); ++x) {
                const int s = y * f.bw + x;
                if (gob[s] > g) h = std::max(h, f.height[s] + 1);
            }
        f.height[b] = h;
    }
}

void level_claims(const std::vector<FrameDepths> &frames, std::vector<int2> &items,
                  std::vector<int> &level_start) {
    int n_levels = 0;
    size_t total = 0;
    for (const FrameDepths &f : frames) {
        total += f.n;
        for (int j = 0; j < f.n; ++j) n_levels = std::max(n_levels, f.level[f.ids[j]] + 1);
    }
    // counting sort by level; within a level by frame, then group order
    level_start.assign(n_levels + 1, 0);
    for (const FrameDepths &f : frames)
        for (int j = 0; j < f.n; ++j) ++level_start[f.level[f.ids[j]] + 1];
    for (int l = 0; l < n_levels; ++l) level_start[l + 1] += level_start[l];
    std::vector<int> fill(level_start.begin(), level_start.end() - 1);
    items.assign(total, make_int2(0, 0));
    for (size_t i = 0; i < frames.size(); ++i) {
        const FrameDepths &f = frames[i];
        for (int j = 0; j < f.n; ++j) {
            const int b = f.ids[j];
            items[fill[f.level[b]]++] = make_int2((int)i, b);
        }
    }
}

namespace {

struct Ready {
    int32_t h, frame, pos, block;
    // priority: longer chain, then earlier frame, then earlier in group order
    bool operator<(const Ready &o) const {
        if (h != o.h) return h < o.h;
        if (frame != o.frame) return frame > o.frame;
        return pos > o.pos;
    }
};

}  // namespace

void schedule_claims(std::vector<FrameDepths> &frames, int rad, int workers,
                     std::vector<int2> &items) {
    std::priority_queue<Ready> ready;
    size_t total = 0;
    for (size_t i = 0; i < frames.size(); ++i) {
        FrameDepths &f = frames[i];
        total += f.n;
        for (int j = 0; j < f.n; ++j) {
            const int b = f.ids[j];
            if (f.indeg[b] == 0) ready.push(Ready{f.height[b], (int32_t)i, j, b});
        }
    }
    items.clear();
    items.reserve(total);
    const size_t P = (size_t)std::max(workers, 1);
    std::vector<Ready> released;
    while (!ready.empty()) {
        released.clear();
        for (size_t t = 0; t < P && !ready.empty(); ++t) {
            const Ready r = ready.top();
            ready.pop();
            items.push_back(make_int2(r.frame, r.block));
            FrameDepths &f = frames[r.frame];
            const int by = r.block / f.bw, bx = r.block - by * f.bw, g = f.gob[r.block];
            for (int y = std::max(0, by - rad); y <= std::min(f.bh - 1, by + rad); ++y)
                for (int x = std::max(0, bx - rad); x <= std::min(f.bw - 1, bx + rad); ++x) {
                    const int s = y * f.bw + x;
                    if (f.gob[s] > g && --f.indeg[s] == 0)
                        released.push_back(Ready{f.height[s], r.frame, f.pos[s], s});
                }
        }
        for (const Ready &r : released) ready.push(r);
    }
}

}  // namespace fse

extern "C" int fse_plan_claims(int n_frames, const int32_t *bw, const int32_t *bh,
                               const int32_t *group_of_block, int block, int workers, int mode,
                               int32_t *items, int32_t *level_start, int32_t *n_levels) {
    using namespace fse;
    const int lb = block_log2(block);
    if (n_frames <= 0 || !bw || !bh || !group_of_block || !items || lb < 0 ||
        (mode != 0 && mode != 1) || (mode == 0 && (!level_start || !n_levels)) ||
        (mode == 1 && workers <= 0))
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
    } else {
        schedule_claims(frames, kBorder >> lb, workers, out);
    }
    for (size_t k = 0; k < out.size(); ++k) {
        items[2 * k] = out[k].x;
        items[2 * k + 1] = out[k].y;
    }
    return FSE_OK;
}
