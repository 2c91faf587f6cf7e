"""Claim order of the executors (host logic, no GPU): one launch per
dependency level, or the list schedule of the persistent CTAs.  A lost block
depends on the earlier-group lost blocks within its area footprint
(+-16/B blocks), whose concealed samples it reads as class R (Sec. 2, 3)."""
import heapq

import numpy as np
import pytest

import fse_synth

fse = pytest.importorskip("paper_2207_00233_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_00233_gb300 import build
    build.build()


def _deps(gob, rad):
    bh, bw = gob.shape
    out = {}
    for by, bx in np.argwhere(gob >= 0):
        g = gob[by, bx]
        d = []
        for y in range(max(0, by - rad), min(bh, by + rad + 1)):
            for x in range(max(0, bx - rad), min(bw, bx + rad + 1)):
                if 0 <= gob[y, x] < g:
                    d.append(y * bw + x)
        out[by * bw + bx] = d
    return out


def _frames(seed, n=3, bh=9, bw=13, B=16):
    rng = np.random.default_rng(seed)
    maps = []
    for i in range(n):
        lost = fse_synth.mixed_block_mask(bh, bw, 0.3 + 0.1 * i, rng).astype(np.uint8)
        gob, _, _ = fse.fse_plan_order(lost, fse.FSE_ORDER_OPTIMIZED)
        maps.append(gob)
    return maps


@pytest.mark.parametrize("B", [16, 8, 4, 2])
def test_levels_are_independent_sets_in_dependency_order(B):
    rad = 16 // B
    maps = _frames(10 + B)
    items, ls = fse.fse_plan_claims(maps, block=B, mode=0)
    deps = [_deps(g, rad) for g in maps]
    # a permutation of the lost blocks
    want = sorted((f, b) for f, g in enumerate(maps) for b in np.flatnonzero(g.ravel() >= 0))
    assert sorted(map(tuple, items.tolist())) == want
    assert ls[0] == 0 and ls[-1] == len(items)
    level = {}
    for l in range(len(ls) - 1):
        for f, b in items[ls[l]:ls[l + 1]]:
            level[(f, b)] = l
    for (f, b), l in level.items():
        # exactly 1 + the deepest dependency: dependencies come in earlier
        # launches and nothing in the same launch depends on another
        assert l == 1 + max((level[(f, d)] for d in deps[f][b]), default=-1)


def _list_schedule(maps, rad, P):
    """Rounds of up to P starts; ready blocks by longest chain of dependants,
    ties first-ready-first (initially frame by frame in group order, then in
    order of release, neighbours scanned row by row); dependants of a round
    become ready in the next one."""
    deps = [_deps(g, rad) for g in maps]
    indeg, height = {}, {}
    buckets = {}
    for f, g in enumerate(maps):
        bh, bw = g.shape
        gf = g.ravel()
        order = sorted(deps[f], key=lambda b: (gf[b], b))
        for b in order:
            indeg[(f, b)] = len(deps[f][b])
        for b in reversed(order):
            by, bx = divmod(b, bw)
            h = 1
            for y in range(max(0, by - rad), min(bh, by + rad + 1)):
                for x in range(max(0, bx - rad), min(bw, bx + rad + 1)):
                    s = y * bw + x
                    if gf[s] > gf[b]:
                        h = max(h, height[(f, s)] + 1)
            height[(f, b)] = h
        for b in order:
            if indeg[(f, b)] == 0:
                buckets.setdefault(height[(f, b)], []).append((f, b))
    out = []
    while True:
        rel = []
        for _ in range(P):
            ready = [h for h, q in buckets.items() if q]
            if not ready:
                break
            f, b = buckets[max(ready)].pop(0)
            out.append((f, b))
            g = maps[f]
            bh, bw = g.shape
            gf = g.ravel()
            by, bx = divmod(b, bw)
            for y in range(max(0, by - rad), min(bh, by + rad + 1)):
                for x in range(max(0, bx - rad), min(bw, bx + rad + 1)):
                    s = y * bw + x
                    if gf[s] > gf[b]:
                        indeg[(f, s)] -= 1
                        if indeg[(f, s)] == 0:
                            rel.append((f, s))
        if not rel and not any(buckets.values()):
            return out
        for k in rel:
            buckets.setdefault(height[k], []).append(k)


@pytest.mark.parametrize("B,P", [(16, 5), (16, 64), (8, 7), (2, 16)])
def test_schedule_matches_list_scheduling(B, P):
    maps = _frames(20 + B, n=2, bh=7, bw=11)
    items, ls = fse.fse_plan_claims(maps, block=B, workers=P, mode=1)
    assert ls is None
    assert [tuple(t) for t in items.tolist()] == _list_schedule(maps, 16 // B, P)


def test_schedule_is_topological_on_a_full_hd_frame():
    img, mask = fse_synth.workload_batch_1080p(1)[0]
    bh, bw = (img.shape[0] + 15) // 16, (img.shape[1] + 15) // 16
    pm = np.zeros((bh * 16, bw * 16), np.uint8)
    pm[:img.shape[0], :img.shape[1]] = mask
    lost = (pm.reshape(bh, 16, bw, 16).max(axis=(1, 3)) > 0).astype(np.uint8)
    gob, _, _ = fse.fse_plan_order(lost, fse.FSE_ORDER_OPTIMIZED)
    items, _ = fse.fse_plan_claims([gob], block=16, workers=456, mode=1)
    seen = np.zeros(bh * bw, bool)
    deps = _deps(gob, 1)
    for _, b in items:
        assert all(seen[d] for d in deps[b])
        seen[b] = True
    assert seen.sum() == (gob >= 0).sum()


def test_single_level_without_dependencies():
    gob = np.full((4, 5), -1, np.int32)
    gob[0, 0] = 0
    gob[3, 4] = 2  # far apart: independent
    items, ls = fse.fse_plan_claims([gob], mode=0)
    assert ls.tolist() == [0, 2] and sorted(items[:, 1].tolist()) == [0, 19]
    none = np.full((2, 2), -1, np.int32)
    items, ls = fse.fse_plan_claims([none], mode=0)
    assert len(items) == 0 and ls.tolist() == [0]


def test_invalid_arguments():
    gob = np.zeros((2, 2), np.int32)
    with pytest.raises(fse.FseError):
        fse.fse_plan_claims([gob], block=3)
    with pytest.raises(fse.FseError):
        fse.fse_plan_claims([gob], mode=3)
    with pytest.raises(fse.FseError):
        fse.fse_plan_claims([gob], mode=1, workers=0)


def _heights(gob, rad):
    bh, bw = gob.shape
    gf = gob.ravel()
    order = sorted(np.flatnonzero(gf >= 0), key=lambda b: (gf[b], b))
    h = {}
    for b in reversed(order):
        by, bx = divmod(int(b), bw)
        v = 1
        for y in range(max(0, by - rad), min(bh, by + rad + 1)):
            for x in range(max(0, bx - rad), min(bw, bx + rad + 1)):
                s = y * bw + x
                if gf[s] > gf[b]:
                    v = max(v, h[s] + 1)
        h[int(b)] = v
    return h, order


@pytest.mark.parametrize("B", [16, 4])
def test_height_order_is_topological_longest_chain_first(B):
    rad = 16 // B
    maps = _frames(40 + B, n=3, bh=8, bw=12)
    items, ls = fse.fse_plan_claims(maps, block=B, mode=2)
    assert ls is None
    want = []
    for f, g in enumerate(maps):
        h, order = _heights(g, rad)
        want += [(-h[b], f, j, int(b)) for j, b in enumerate(order)]
    want.sort()
    assert [tuple(t) for t in items.tolist()] == [(f, b) for _, f, _, b in want]
    # dependencies first
    deps = [_deps(g, rad) for g in maps]
    seen = set()
    for f, b in items.tolist():
        assert all((f, d) in seen for d in deps[f][b])
        seen.add((f, b))


@pytest.mark.parametrize("B,P", [(16, 5), (16, 40), (4, 16)])
def test_delayed_height_order(B, P):
    """Mode 3 (the persistent executor's order): the height order in rounds
    of P claims, each block raised to one past its latest dependency's round,
    sorted by round, then frame, then group order."""
    rad = 16 // B
    maps = _frames(60 + B, n=3, bh=8, bw=12)
    hitems, _ = fse.fse_plan_claims(maps, block=B, mode=2)
    items, ls = fse.fse_plan_claims(maps, block=B, workers=P, mode=3)
    assert ls is None
    deps = [_deps(g, rad) for g in maps]
    key = {(int(f), int(b)): pos // P for pos, (f, b) in enumerate(hitems.tolist())}
    for f, g in enumerate(maps):
        gf = g.ravel()
        for b in sorted(deps[f], key=lambda b: (gf[b], b)):
            key[(f, b)] = max([key[(f, b)]] + [key[(f, d)] + 1 for d in deps[f][b]])
    gpos = {}
    for f, g in enumerate(maps):
        gf = g.ravel()
        for j, b in enumerate(sorted(np.flatnonzero(gf >= 0), key=lambda b: (gf[b], b))):
            gpos[(f, int(b))] = j
    want = sorted((key[k], k[0], gpos[k], k[1]) for k in key)
    assert [tuple(t) for t in items.tolist()] == [(f, b) for _, f, _, b in want]
    seen = set()
    for f, b in items.tolist():
        assert all((f, d) in seen for d in deps[f][b])
        seen.add((f, b))
