"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
DFT, closed forms, brute force on tiny areas, invariants, or hand-derived
golden schedules (Sec. 2 Eq. (1)-(2), Sec. 3 Algorithm 1, Sec. 4 parameters).
"""
import os

import numpy as np
import pytest

import fse_synth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _phi(F, M, N, k):
    km, kn = divmod(int(k), F)
    mm, nn = np.mgrid[0:M, 0:N]
    return np.exp(2j * np.pi * (km * mm + kn * nn) / F)


def _model(F, M, N, u, dc, upto=None):
    g = np.zeros((M, N), complex)
    for i in range(len(u) if upto is None else upto):
        g += dc[i] * _phi(F, M, N, u[i])
    return g


def _random_area(M, N, seed, lost=((2, 4), (2, 4)), recon=None):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0, 255, (M, N))
    cls = np.zeros((M, N), np.uint8)
    (a, b), (c, d) = lost
    cls[a:b, c:d] = oracle.CLS_BI
    if recon is not None:
        (a, b), (c, d) = recon
        cls[a:b, c:d] = oracle.CLS_R
    return f, cls


# --------------------------------------------------------------------------
# Transform: the initial projection is the zero-extended 2-D DFT (Sec. 4).
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,F", [(6, 6, 8), (5, 7, 8), (12, 10, 16), (48, 48, 64)])
def test_projection_equals_library_dft(M, N, F):
    f, cls = _random_area(M, N, 1, lost=((1, 3), (2, 5)), recon=((0, 1), (0, 3)))
    r = oracle.extrapolate_area(f, cls, F, 0, 0.7, 0.2, 0.5)
    x = np.zeros((F, F))
    x[:M, :N] = r.w * f
    wp = np.zeros((F, F))
    wp[:M, :N] = r.w
    scale = np.abs(np.fft.fft2(x)).max()
    assert np.abs(r.R0 - np.fft.fft2(x)).max() <= 1e-12 * scale
    assert np.abs(r.W - np.fft.fft2(wp)).max() <= 1e-12 * np.abs(r.W).max()
    # Real input: the spectrum is exactly conjugate symmetric (ties are exact).
    neg = (-np.arange(F)) % F
    assert np.array_equal(r.R0[np.ix_(neg, neg)], np.conj(r.R0))


# --------------------------------------------------------------------------
# Weighting function, Eq. (2).
# --------------------------------------------------------------------------

def test_weights_closed_form_3x3():
    rho, delta = 0.6, 0.25
    cls = np.full((3, 3), oracle.CLS_A, np.uint8)
    w = oracle.weights(cls, rho, delta)
    # centre ((M-1)/2, (N-1)/2) = (1, 1): distance 0, 1 and sqrt(2)
    assert w[1, 1] == 1.0
    for (m, n) in [(0, 1), (1, 0), (1, 2), (2, 1)]:
        assert w[m, n] == pytest.approx(0.6, rel=1e-15)
    for (m, n) in [(0, 0), (0, 2), (2, 0), (2, 2)]:
        assert w[m, n] == pytest.approx(0.6 ** np.sqrt(2.0), rel=1e-15)
    cls2 = cls.copy()
    cls2[0, 1] = oracle.CLS_R
    cls2[2, 2] = oracle.CLS_BI
    cls2[0, 0] = oracle.CLS_BO
    cls2[1, 0] = oracle.CLS_OUT
    w2 = oracle.weights(cls2, rho, delta)
    assert w2[0, 1] == pytest.approx(0.25 * 0.6, rel=1e-15)
    assert w2[2, 2] == 0.0 and w2[0, 0] == 0.0 and w2[1, 0] == 0.0


def test_weights_even_size_centre_and_symmetry():
    rho = 0.7
    cls = np.zeros((48, 48), np.uint8)
    w = oracle.weights(cls, rho, 0.2)
    # centre at (23.5, 23.5): the four middle samples are at distance sqrt(0.5)
    assert w[23, 23] == pytest.approx(rho ** np.sqrt(0.5), rel=1e-15)
    assert np.array_equal(w, w[::-1, :]) and np.array_equal(w, w[:, ::-1])
    assert np.array_equal(w, w.T)
    # decreasing with distance along a row through the middle
    assert np.all(np.diff(w[23, 24:]) < 0)


# --------------------------------------------------------------------------
# Iteration: selection, compensated coefficient, residual update.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_final_residual_equals_spatial_definition(seed):
    """R_w after K iterations = DFT{w (f - g)} with g = sum dc_i phi_{u_i}."""
    M = N = 12
    F = 16
    f, cls = _random_area(M, N, seed, lost=((4, 8), (4, 8)), recon=((0, 2), (0, 12)))
    K = 30
    r = oracle.extrapolate_area(f, cls, F, K, 0.7, 0.2, 0.5)
    g = _model(F, M, N, r.u, r.dc)
    x = np.zeros((F, F), complex)
    x[:M, :N] = r.w * (f - g)
    ref = np.fft.fft2(x)
    assert np.abs(r.R - ref).max() <= 1e-10 * np.abs(r.R0).max()
    # the dense coefficients are the accumulated increments
    coef = np.zeros(F * F, complex)
    np.add.at(coef, r.u, r.dc)
    assert np.allclose(r.coef.ravel(), coef, rtol=0, atol=1e-12 * np.abs(coef).max())
    # the returned model is the real part of Eq. (1)
    assert np.abs(r.g - g.real).max() <= 1e-9 * np.abs(f).max()


@pytest.mark.parametrize("seed", [3, 4])
def test_energy_decrease_closed_form_and_monotone(seed):
    M = N = 10
    F = 16
    gamma = 0.5
    f, cls = _random_area(M, N, seed, lost=((3, 7), (3, 7)))
    K = 25
    r = oracle.extrapolate_area(f, cls, F, K, 0.8, 0.2, gamma)
    W0 = r.w.sum()
    E = []
    for nu in range(K + 1):
        res = f - _model(F, M, N, r.u, r.dc, upto=nu)
        E.append(np.sum(r.w * np.abs(res) ** 2))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-9 * E[0])
    # |R_w[u]| at selection time equals |dc| W0 / gamma; the energy drops by
    # (2 gamma - gamma^2) |R_w[u]|^2 / W0
    pred = (2 * gamma - gamma ** 2) * (np.abs(r.dc) * W0 / gamma) ** 2 / W0
    assert np.allclose(E[:-1] - E[1:], pred, rtol=1e-8, atol=1e-9 * E[0])


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_selection_matches_spatial_brute_force(seed):
    """On a 6x6 area with an 8x8 DFT every iteration's choice maximises the
    spatial weighted-energy decrease over all 64 basis functions."""
    M = N = 6
    F = 8
    gamma = 0.5
    f, cls = _random_area(M, N, seed, lost=((2, 4), (2, 4)), recon=((0, 1), (0, 6)))
    K = 12
    r = oracle.extrapolate_area(f, cls, F, K, 0.7, 0.2, gamma)
    w = r.w
    W0 = w.sum()
    phis = [_phi(F, M, N, k) for k in range(F * F)]
    res = f.astype(complex)
    for nu in range(K):
        E = np.sum(w * np.abs(res) ** 2)
        dE = np.empty(F * F)
        for k in range(F * F):
            p = np.sum(w * res * np.conj(phis[k])) / W0
            dE[k] = E - np.sum(w * np.abs(res - gamma * p * phis[k]) ** 2)
        best = dE.max()
        near = np.flatnonzero(dE >= best * (1 - 1e-9))
        assert r.u[nu] == near.min(), (nu, r.u[nu], near)
        p = np.sum(w * res * np.conj(phis[r.u[nu]])) / W0
        assert abs(r.dc[nu] - gamma * p) <= 1e-9 * abs(p)
        res = res - r.dc[nu] * phis[r.u[nu]]


def test_constant_support_is_reproduced():
    M = N = 48
    F = 64
    f = np.full((M, N), 93.0)
    cls = np.zeros((M, N), np.uint8)
    cls[16:32, 16:32] = oracle.CLS_BI
    cls[0:16, 0:48] = oracle.CLS_BO
    r = oracle.extrapolate_area(f, cls, F, 100, 0.7, 0.2, 0.5)
    assert np.abs(r.g[16:32, 16:32] - 93.0).max() <= 1e-9


@pytest.mark.parametrize("a,b,phase", [(3, 5, 0.3), (0, 4, 1.1), (10, 3, -0.7), (7, 60, 2.0)])
def test_on_grid_cosine_is_extrapolated_exactly(a, b, phase):
    M = N = 48
    F = 64
    mm, nn = np.mgrid[0:M, 0:N]
    f = 100 + 50 * np.cos(2 * np.pi * (a * mm + b * nn) / F + phase)
    cls = np.zeros((M, N), np.uint8)
    cls[16:32, 16:32] = oracle.CLS_BI
    r = oracle.extrapolate_area(f, cls, F, 200, 0.7, 0.2, 0.5)
    assert np.abs(r.g - f)[16:32, 16:32].max() <= 1e-6


def test_scaling_homogeneity():
    M = N = 48
    F = 64
    f, cls = _random_area(M, N, 11, lost=((16, 32), (16, 32)), recon=((0, 16), (0, 48)))
    r1 = oracle.extrapolate_area(f, cls, F, 60, 0.7, 0.2, 0.5)
    r2 = oracle.extrapolate_area(2.0 * f, cls, F, 60, 0.7, 0.2, 0.5)
    assert np.array_equal(r2.g, 2.0 * r1.g)          # power of two: exact
    assert np.array_equal(r2.u, r1.u)
    r3 = oracle.extrapolate_area(0.37 * f, cls, F, 60, 0.7, 0.2, 0.5)
    assert np.abs(r3.g - 0.37 * r1.g).max() <= 1e-9 * np.abs(r1.g).max()


def test_conjugate_tie_break_gives_same_real_model():
    """Real input gives exact ties between k and -k; choosing the mirror
    member yields the conjugate-mirror trajectory and the same real part."""
    M = N = 48
    F = 64
    _, cls = _random_area(M, N, 12, lost=((16, 32), (16, 32)))
    rng = np.random.default_rng(12)
    mm, nn = np.mgrid[0:M, 0:N]
    f = 80 * np.cos(2 * np.pi * (5 * mm + 3 * nn) / F + 0.3) + rng.normal(0, 20, (M, N))
    r1 = oracle.extrapolate_area(f, cls, F, 100, 0.7, 0.2, 0.5, tie_largest=False)
    r2 = oracle.extrapolate_area(f, cls, F, 100, 0.7, 0.2, 0.5, tie_largest=True)
    assert r1.u[0] != r2.u[0]
    neg = lambda k: ((-(k // F)) % F) * F + ((-(k % F)) % F)
    assert r2.u[0] == neg(r1.u[0])
    assert np.abs(r1.g - r2.g)[16:32, 16:32].max() <= 1e-9


def test_no_support_gives_zero_model():
    f = np.full((8, 8), 50.0)
    cls = np.full((8, 8), oracle.CLS_BO, np.uint8)
    r = oracle.extrapolate_area(f, cls, 8, 10, 0.7, 0.2, 0.5)
    assert np.all(r.g == 0.0) and np.all(r.u == -1)


# --------------------------------------------------------------------------
# Processing order, Algorithm 1 (Sec. 3).
# --------------------------------------------------------------------------

def _load_grid(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("grid"):
                continue
            rows.append([int(t) for t in line.split()])
    return np.array(rows, np.int32)


@pytest.mark.parametrize("name", ["schedule_5x5_centre.txt", "schedule_8x8_row.txt",
                                  "schedule_3x3_all.txt"])
def test_schedule_golden(name):
    want = _load_grid(name)
    lost = (want >= 0).astype(np.uint8)
    gob, gptr, ids = oracle.plan(lost, oracle.ORDER_OPTIMIZED)
    assert np.array_equal(gob, want)
    assert len(gptr) - 1 == want.max() + 1


def _check_schedule_invariants(lost, gob, gptr, ids):
    bh, bw = lost.shape
    assert np.array_equal(gob < 0, lost == 0)
    assert sorted(ids.tolist()) == np.flatnonzero(lost.ravel()).tolist()
    for g in range(len(gptr) - 1):
        members = ids[gptr[g]:gptr[g + 1]]
        assert len(members) > 0
        assert np.all(np.diff(members) > 0)          # raster order inside a group
        for b in members:
            by, bx = divmod(int(b), bw)
            assert gob[by, bx] == g
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dy == dx == 0:
                        continue
                    ny, nx = by + dy, bx + dx
                    if 0 <= ny < bh and 0 <= nx < bw:
                        assert gob[ny, nx] != g      # independent under 8-adjacency


@pytest.mark.parametrize("seed", range(20))
def test_schedule_invariants_random(seed):
    rng = np.random.default_rng(seed)
    bh, bw = int(rng.integers(1, 14)), int(rng.integers(1, 14))
    lost = (rng.random((bh, bw)) < rng.uniform(0.05, 0.95)).astype(np.uint8)
    gob, gptr, ids = oracle.plan(lost, oracle.ORDER_OPTIMIZED)
    _check_schedule_invariants(lost, gob, gptr, ids)
    assert len(gptr) - 1 <= int(lost.sum())
    gob0, gptr0, ids0 = oracle.plan(lost, oracle.ORDER_LINESCAN)
    assert np.array_equal(ids0, np.flatnonzero(lost.ravel()))
    assert np.array_equal(np.diff(gptr0), np.ones(int(lost.sum()), np.int32))


def test_isolated_losses_form_one_group():
    lost = np.zeros((9, 9), np.uint8)
    lost[1::3, 1::3] = 1
    gob, gptr, ids = oracle.plan(lost, oracle.ORDER_OPTIMIZED)
    assert len(gptr) == 2 and np.all(gob[lost == 1] == 0)


# --------------------------------------------------------------------------
# Whole frame.
# --------------------------------------------------------------------------

def test_no_loss_frame_is_unchanged():
    img = fse_synth.make_image(64, 80, 5)
    mask = np.zeros_like(img)
    work, out, gob = oracle.conceal_frame(img, mask, iters=20)
    assert np.array_equal(out, img) and np.array_equal(work, img.astype(np.float64))
    assert np.all(gob == -1)


def test_constant_frame_is_restored_exactly():
    img = np.full((80, 96), 77, np.uint8)
    rng = np.random.default_rng(3)
    lost = (rng.random((5, 6)) < 0.4).astype(np.uint8)
    mask = fse_synth.blocks_to_pixel_mask(lost, 80, 96)
    for order in (0, 1):
        work, out, _ = oracle.conceal_frame(img, mask, iters=100, order=order)
        assert np.array_equal(out, img)
        assert np.abs(work - 77.0).max() <= 1e-6


def test_smooth_frame_is_extrapolated_accurately():
    """A low-frequency on-grid cosine image (8-bit rounded) is concealed to
    within a few 8-bit steps in every lost block, whatever the order."""
    H, W = 96, 112
    yy, xx = np.mgrid[0:H, 0:W]
    truth = 128 + 60 * np.cos(2 * np.pi * (3 * yy + 5 * xx) / 64 + 0.4)
    img = np.rint(truth).astype(np.uint8)
    rng = np.random.default_rng(9)
    lost = (rng.random((6, 7)) < 0.35).astype(np.uint8)
    lost[2, 1:5] = 1
    mask = fse_synth.blocks_to_pixel_mask(lost, H, W)
    for order in (0, 1):
        work, out, _ = oracle.conceal_frame(img, mask, iters=200, order=order)
        err = np.abs(work - truth)[mask == 1]
        assert err.max() <= 3.0, (order, err.max())
        assert np.sqrt(np.mean(err ** 2)) <= 1.0


def test_isolated_losses_same_for_both_orders():
    """Isolated 16x16 losses: both orders give the identical frame
    (Table 1, isolated 16x16 row)."""
    img = fse_synth.make_image(128, 128, 21)
    lost = np.zeros((8, 8), np.uint8)
    lost[1::3, 1::3] = 1
    lost[6, 0] = 1
    mask = fse_synth.blocks_to_pixel_mask(lost, 128, 128)
    w0, o0, _ = oracle.conceal_frame(img, mask, iters=50, order=0)
    w1, o1, _ = oracle.conceal_frame(img, mask, iters=50, order=1)
    assert np.array_equal(w0, w1) and np.array_equal(o0, o1)


def test_partial_edge_blocks_and_threads_agree():
    img = fse_synth.make_image(40, 56, 8)             # 3x4 blocks, partial last row/col
    rng = np.random.default_rng(8)
    lost = (rng.random((3, 4)) < 0.5).astype(np.uint8)
    lost[2, 3] = 1
    mask = fse_synth.blocks_to_pixel_mask(lost, 40, 56)
    w1, o1, _ = oracle.conceal_frame(img, mask, iters=40, threads=1)
    w4, o4, _ = oracle.conceal_frame(img, mask, iters=40, threads=4)
    assert np.array_equal(w1, w4) and np.array_equal(o1, o4)
    assert np.array_equal(o1[mask == 0], img[mask == 0])
    assert np.all(w1[mask == 1] >= 0) and np.all(w1[mask == 1] <= 255)


def test_fully_lost_single_block_frame():
    img = np.full((16, 16), 200, np.uint8)
    mask = np.ones_like(img)
    work, out, gob = oracle.conceal_frame(img, mask, iters=10)
    assert np.all(out == 0) and gob[0, 0] == 0
