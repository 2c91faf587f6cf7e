"""Pins of the oracle's frame-level sub-area classes and group snapshot.

Sec. 2 (Fig. 1) splits the extrapolation area of a block into the support A
(samples never lost), the reconstructed area R (lost samples of blocks that
were concealed before), the block itself B_i and the lost samples of blocks
still to come, B_o.  Sec. 3 (Algorithm 1) conceals the blocks of one group
"in parallel": every block of a group reads the frame as it was when the
group started, so a block of the same group is never R, whatever the scan
order inside the group.

The expected class grids below are written out by hand from the golden
schedules (one symbol per neighbour block of the area) and are not computed
by any code that mirrors the oracle's classification.  Each pin fails if R
is read as B_o, if a block of the same group is read as R, or if a block's
own samples or the support are mislabelled.  The last two tests recompute a
concealed block from a hand-built area through the oracle's area function
and require the frame result to match exactly: that fixes the values the
frame feeds in for R (the concealed samples, weighted delta * rho^dist by
Eq. (2)) and for A (the image).
"""
import numpy as np
import pytest

import fse_synth
import oracle

A, R, BI, BO, OUT = oracle.CLS_A, oracle.CLS_R, oracle.CLS_BI, oracle.CLS_BO, oracle.CLS_OUT
_SYM = {"A": A, "R": R, "I": BI, "O": BO, "X": OUT}


def _expand(table, B):
    """A hand-written table of neighbour-block classes (rows of symbols:
    A, R, I = B_i, O = B_o, X = outside the image) -> per-sample classes."""
    rows = [[_SYM[t] for t in row.split()] for row in table]
    return np.kron(np.array(rows, np.uint8), np.ones((B, B), np.uint8))


def _block_mask(lost, B):
    return np.kron(lost.astype(np.uint8), np.ones((B, B), np.uint8))


# ---------------------------------------------------------------------------
# 5x5 blocks of 16x16, the centre 3x3 lost (golden schedule:
# groups 0 = corners of the square, 1 = (1,2), (3,2), 2 = (2,1), (2,3),
# 3 = centre).  With d = 16 the area is the block and its 8 neighbours.
# ---------------------------------------------------------------------------

_CENTRE_5X5 = {
    (2, 2): ["R R R",
             "R I R",
             "R R R"],          # group 3: all eight neighbours concealed before
    (1, 2): ["A A A",
             "R I R",            # corners (1,1), (1,3): group 0, concealed
             "O O O"],           # (2,1), (2,3): group 2; (2,2): group 3
    (1, 1): ["A A A",
             "A I O",            # (1,2): group 1, later
             "A O O"],
    (2, 1): ["A R R",            # (1,1) group 0, (1,2) group 1: both earlier
             "A I O",            # (2,2): group 3
             "A R R"],
    (3, 2): ["O O O",
             "R I R",
             "A A A"],
}


def _frame_5x5(seed=31):
    img = fse_synth.make_image(80, 80, seed)
    lost = np.zeros((5, 5), np.uint8)
    lost[1:4, 1:4] = 1
    return img, _block_mask(lost, 16)


@pytest.mark.parametrize("block", sorted(_CENTRE_5X5))
def test_classes_centre_square(block):
    img, mask = _frame_5x5()
    _, _, gob, cls = oracle.conceal_frame(img, mask, iters=20, order=oracle.ORDER_OPTIMIZED,
                                          classes=True)
    want = _expand(_CENTRE_5X5[block], 16)
    by, bx = block
    assert np.array_equal(cls[by * 5 + bx], want), block


def test_classes_image_corner_and_linescan():
    """Corner block of a 3x3 all-lost frame: the area rows and columns that
    fall outside the image are their own class.  Line scan conceals one
    block at a time, so every earlier block in raster order is R."""
    img = fse_synth.make_image(48, 48, 32)
    mask = np.ones((48, 48), np.uint8)
    # Algorithm 1 golden (3x3 all lost): (0,0) is in group 0, (1,1) in group 1
    _, _, _, cls = oracle.conceal_frame(img, mask, iters=10, order=oracle.ORDER_OPTIMIZED,
                                        classes=True)
    assert np.array_equal(cls[0], _expand(["X X X",
                                           "X I O",
                                           "X O O"], 16))
    assert np.array_equal(cls[4], _expand(["R O R",     # (0,1) group 2, (1,0) group 3
                                           "O I O",
                                           "R O R"], 16))
    _, _, _, cls = oracle.conceal_frame(img, mask, iters=10, order=oracle.ORDER_LINESCAN,
                                        classes=True)
    assert np.array_equal(cls[4], _expand(["R R R",
                                           "R I O",
                                           "O O O"], 16))
    assert np.array_equal(cls[8], _expand(["R R X",
                                           "R I X",
                                           "X X X"], 16))


# ---------------------------------------------------------------------------
# Block size 8 with d = 16 (40x40 area, +-2 blocks): blocks of one group can
# lie inside each other's area.  6 x 8 blocks of 8x8; lost (2,1), (2,3),
# (2,5), (3,3), (4,3).  Algorithm 1 by hand: N = 0 for (2,1) and (2,5), 1 for
# (2,3) and (4,3) (their neighbour (3,3)), 2 for (3,3); rounds: {(2,1),
# (2,5)}, {(2,3), (4,3)} (not adjacent: two rows apart), {(3,3)}.
# ---------------------------------------------------------------------------

def _frame_b8(seed=33):
    img = fse_synth.make_image(48, 64, seed)
    lost = np.zeros((6, 8), np.uint8)
    for b in [(2, 1), (2, 3), (2, 5), (3, 3), (4, 3)]:
        lost[b] = 1
    return img, _block_mask(lost, 8), lost


_B8 = {
    (2, 3): ["A A A A A",
             "A A A A A",
             "R A I A R",        # (2,1), (2,5): group 0
             "A A O A A",        # (3,3): group 2
             "A A O A A"],       # (4,3): group 1, same group -> not yet concealed
    (4, 3): ["R A O A R",        # (2,3): same group (snapshot) -> B_o
             "A A O A A",
             "A A I A A",
             "A A A A A",
             "X X X X X"],       # block row 6 is outside the 6-row grid
    (3, 3): ["A A A A A",
             "R A R A R",
             "A A I A A",
             "A A R A A",
             "A A A A A"],
}


def test_b8_schedule_by_hand():
    _, _, lost = _frame_b8()
    gob, _, _ = oracle.plan(lost, oracle.ORDER_OPTIMIZED)
    want = np.full((6, 8), -1, np.int32)
    want[2, 1] = want[2, 5] = 0
    want[2, 3] = want[4, 3] = 1
    want[3, 3] = 2
    assert np.array_equal(gob, want)


@pytest.mark.parametrize("block", sorted(_B8))
def test_classes_b8_group_snapshot(block):
    img, mask, _ = _frame_b8()
    _, _, _, cls = oracle.conceal_frame(img, mask, block=8, border=16, iters=20,
                                        order=oracle.ORDER_OPTIMIZED, classes=True)
    by, bx = block
    assert np.array_equal(cls[by * 8 + bx], _expand(_B8[block], 8)), block


def _area_values(img, work, top, left, cls):
    """f of a hand-classified area: image samples for A, concealed samples
    for R, zero elsewhere."""
    M = cls.shape[0]
    H, W = img.shape
    f = np.zeros((M, M))
    for m in range(M):
        for n in range(M):
            y, x = top + m, left + n
            if cls[m, n] == A:
                f[m, n] = img[y, x]
            elif cls[m, n] == R:
                f[m, n] = work[y, x]
    return f


def _recompute(img, work, block, table, B, K, rho, delta, gamma):
    by, bx = block
    cls = _expand(table, B)
    f = _area_values(img, work, by * B - 16, bx * B - 16, cls)
    r = oracle.extrapolate_area(f, cls, 64, K, rho, delta, gamma)
    return np.clip(r.g[16:16 + B, 16:16 + B], 0.0, 255.0), f, cls


@pytest.mark.parametrize("block", [(1, 2), (2, 1), (3, 2), (2, 2)])
def test_frame_result_equals_hand_built_area(block):
    """A block of a later group, recomputed from a hand-built area (A from
    the image, R from the concealed samples of the earlier groups, classes
    from the table), equals the frame result; the same area with R read as
    B_o, or with the delta factor dropped, does not."""
    img = fse_synth.make_image(80, 80, 34)
    img[16:64, 16:64] = np.clip(img[16:64, 16:64].astype(int) + 90, 0, 255).astype(np.uint8)
    lost = np.zeros((5, 5), np.uint8)
    lost[1:4, 1:4] = 1
    mask = _block_mask(lost, 16)
    K, rho, delta, gamma = 60, 0.7, 0.2, 0.5
    work, _, _ = oracle.conceal_frame(img, mask, iters=K, rho=rho, delta=delta, gamma=gamma,
                                      order=oracle.ORDER_OPTIMIZED)
    by, bx = block
    got = work[by * 16:by * 16 + 16, bx * 16:bx * 16 + 16]
    g, f, cls = _recompute(img, work, block, _CENTRE_5X5[block], 16, K, rho, delta, gamma)
    assert np.abs(g - got).max() <= 1e-12
    # the concealed samples around the square's centre differ from the
    # support outside it (the square is brightened), so R carries information
    assert (cls == R).any()
    as_bo = np.where(cls == R, BO, cls).astype(np.uint8)
    g_bo = np.clip(oracle.extrapolate_area(f, as_bo, 64, K, rho, delta, gamma)
                   .g[16:32, 16:32], 0, 255)
    assert np.abs(g_bo - got).max() > 1.0
    if (cls == A).any():
        # delta weighs R against A (with R alone a common factor cancels)
        as_a = np.where(cls == R, A, cls).astype(np.uint8)
        g_a = np.clip(oracle.extrapolate_area(f, as_a, 64, K, rho, delta, gamma)
                      .g[16:32, 16:32], 0, 255)
        assert np.abs(g_a - got).max() > 1.0


def test_frame_result_b8_snapshot_values():
    """Block (4,3) at B = 8 shares its group with (2,3), which lies in its
    area: the frame result equals the hand-built area in which (2,3) is
    B_o (the group-start snapshot), not the one in which it is R."""
    img, mask, _ = _frame_b8(35)
    K, rho, delta, gamma = 60, 0.7, 0.2, 0.5
    work, _, _ = oracle.conceal_frame(img, mask, block=8, border=16, iters=K, rho=rho,
                                      delta=delta, gamma=gamma, order=oracle.ORDER_OPTIMIZED)
    got = work[32:40, 24:32]
    g, f, cls = _recompute(img, work, (4, 3), _B8[(4, 3)], 8, K, rho, delta, gamma)
    assert np.abs(g - got).max() <= 1e-12
    seq = _B8[(4, 3)].copy()
    seq[0] = "R A R A R"                                   # a sequential reading
    g_seq, _, _ = _recompute(img, work, (4, 3), seq, 8, K, rho, delta, gamma)
    assert np.abs(g_seq - got).max() > 0.5
