"""GPU parity: the sm_103a path against the FP64 oracle, through the C-ABI.

Workloads are the seeded synthetic stand-ins for the paper's test images
(Sec. 4): 128x128 with 10% i.i.d. losses and K = 100 (line scan), 512x512
with 25% mixed isolated/burst losses and K = 200 (both orders), small
frames with partial edge blocks, degenerate frames, and the full-size
16-frame 1920x1080 batch checked on sampled frames.  Blocks whose FP32
selections follow the oracle's are compared sample by sample (|d| <= 0.5,
PSNR >= 50 dB); blocks that diverge at a near-tie are checked for validity
(see gpu_util).
"""
import numpy as np
import pytest

import fse_synth
import oracle
from fse_check import TAU_SCALE, near_tie_at_divergence, trajectory
from gpu_util import gpu_conceal, oracle_conceal, run_and_compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2207_00233_gb300 import build
    build.build()
    import paper_2207_00233_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(fse):
    c = fse.Context(0)
    c.fse_ctx_set_option(fse.FSE_OPT_KEEP_TRACE, 1)
    yield c
    c.close()


EXECS = ["groups", "persistent"]


def _params(fse, iters, order, executor, rho=0.7):
    ex = fse.FSE_EXEC_PERSISTENT if executor == "persistent" else fse.FSE_EXEC_GROUPS
    return fse.make_params(iters=iters, rho=rho, delta=0.2, gamma=0.5, order=order, executor=ex)


@pytest.mark.parametrize("executor", EXECS)
def test_single_128_linescan(fse, ctx, executor):
    frames = fse_synth.workload_single_128()
    p = _params(fse, 100, fse.FSE_ORDER_LINESCAN, executor)
    *_, st = run_and_compare(ctx, frames, p, "128 line scan")
    print(st)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("executor", EXECS)
def test_mixed_512(fse, ctx, order, executor):
    frames = fse_synth.workload_mixed_512()
    p = _params(fse, 200, order, executor)
    *_, st = run_and_compare(ctx, frames, p, f"512 order {order}")
    print(st)
    o_gob = oracle.plan(
        (np.add.reduceat(np.add.reduceat(frames[0][1], np.arange(0, 512, 16), 0),
                         np.arange(0, 512, 16), 1) > 0).astype(np.uint8), order)[0]
    info = ctx.fse_last_batch_info()
    assert info["groups"] == int(o_gob.max()) + 1
    assert info["lost_blocks"] == int((o_gob >= 0).sum())


@pytest.mark.parametrize("order", [0, 1])
def test_mixed_512_split_tf32_projection(fse, ctx, order):
    """The split-TF32 tensor-core projection is FP32-grade: the same parity
    criteria as the FP32 path."""
    frames = fse_synth.workload_mixed_512()
    p = fse.make_params(iters=200, rho=0.7, delta=0.2, gamma=0.5, order=order,
                        executor=fse.FSE_EXEC_PERSISTENT, precision=fse.FSE_PREC_TF32X3)
    *_, st = run_and_compare(ctx, frames, p, f"512 tf32x3 order {order}")
    print(st)


def test_full_size_split_tf32_projection(fse, ctx):
    frames = fse_synth.workload_batch_1080p(16)
    p = fse.make_params(iters=200, order=1, executor=fse.FSE_EXEC_PERSISTENT,
                        precision=fse.FSE_PREC_TF32X3)
    *_, st = run_and_compare(ctx, frames, p, "1080p tf32x3", sample=(0, 5))
    print(st)


@pytest.mark.parametrize("order", [0, 1])
def test_mixed_512_split_bf16_projection(fse, ctx, order):
    """The split-BF16 tensor-core projection (about 16 significant bits per
    operand, so tau uses 2^-16): every selection is a valid maximiser within
    tau, clean blocks match the oracle, and every root is a block whose FP64
    trajectory has a near-tie within that tau."""
    frames = fse_synth.workload_mixed_512()
    p = fse.make_params(iters=200, rho=0.7, delta=0.2, gamma=0.5, order=order,
                        executor=fse.FSE_EXEC_PERSISTENT, precision=fse.FSE_PREC_BF16X3)
    *_, st = run_and_compare(ctx, frames, p, f"512 bf16x3 order {order}")
    print(st)


def test_full_size_split_bf16_projection(fse, ctx):
    frames = fse_synth.workload_batch_1080p(16)
    p = fse.make_params(iters=200, order=1, executor=fse.FSE_EXEC_PERSISTENT,
                        precision=fse.FSE_PREC_BF16X3)
    *_, st = run_and_compare(ctx, frames, p, "1080p bf16x3", sample=(0,))
    print(st)


def test_mixed_512_paper_rho(fse, ctx):
    frames = fse_synth.workload_mixed_512()
    p = _params(fse, 200, fse.FSE_ORDER_OPTIMIZED, "persistent", rho=0.8)
    *_, st = run_and_compare(ctx, frames, p, "512 rho 0.8")
    print(st)


def test_executors_bit_identical(fse, ctx):
    """Launch per dependency level, launch per plan group, and the persistent
    launch read the same samples in every block: identical bytes."""
    img, mask = fse_synth.workload_mixed_512()[0]
    res = []
    for ex, per_group in (("groups", 0), ("groups", 1), ("persistent", 0)):
        ctx.fse_ctx_set_option(fse.FSE_OPT_GROUP_LAUNCHES, per_group)
        p = _params(fse, 200, fse.FSE_ORDER_OPTIMIZED, ex)
        outs, works = gpu_conceal(ctx, [(img, mask)], p)
        res.append((outs[0], works[0], ctx.fse_last_batch_info()))
    ctx.fse_ctx_set_option(fse.FSE_OPT_GROUP_LAUNCHES, 0)
    for o, wk, _ in res[1:]:
        assert np.array_equal(res[0][0], o)
        assert np.array_equal(res[0][1], wk, equal_nan=True)
    # one launch per group (plus the loss map) against fewer per level
    assert res[1][2]["launches"] == res[1][2]["groups"] + 1
    assert res[0][2]["launches"] < res[1][2]["launches"]


@pytest.mark.parametrize("h,w,rate,seed", [(40, 56, 0.5, 1), (100, 70, 0.3, 2),
                                           (16, 16, 1.0, 3), (33, 200, 0.4, 4),
                                           (200, 17, 0.6, 5)])
@pytest.mark.parametrize("order", [0, 1])
def test_small_frames_partial_blocks(fse, ctx, h, w, rate, seed, order):
    frames = [fse_synth.random_frame(h, w, rate, seed)]
    p = _params(fse, 60, order, "persistent")
    run_and_compare(ctx, frames, p, f"{h}x{w}")


@pytest.mark.parametrize("h,w,kind", [(1, 1, "lost"), (5, 7, "random"), (1, 40, "random"),
                                      (40, 1, "random"), (17, 17, "last")])
def test_degenerate_frame_sizes(fse, ctx, h, w, kind):
    """Frames smaller than one block, one sample high or wide, or with a
    single lost sample in a partial corner block, in both orders, against
    the oracle.  A lost 1x1 frame has no support at all: W[0] = 0, so no
    iteration runs and the sample becomes 0, as in the oracle."""
    rng = np.random.default_rng(h * 100 + w)
    img = (rng.random((h, w)) * 255).astype(np.uint8)
    if kind == "random":
        mask = (rng.random((h, w)) < 0.4).astype(np.uint8)
    elif kind == "last":
        mask = np.zeros((h, w), np.uint8)
        mask[-1, -1] = 1
    else:
        mask = np.ones((h, w), np.uint8)
    for order in (0, 1):
        p = _params(fse, 30, order, "persistent")
        run_and_compare(ctx, [(img, mask)], p, f"{h}x{w} {kind} order {order}")


def test_one_sample_frame_without_loss_unchanged(fse, ctx):
    img = np.array([[173]], np.uint8)
    (out,), _ = gpu_conceal(ctx, [(img, np.zeros_like(img))], _params(fse, 30, 1, "persistent"),
                            want_work=False)
    assert np.array_equal(out, img)


def test_empty_batch_rejected(fse, ctx):
    with pytest.raises(fse.FseError):
        ctx.fse_conceal_batch([], _params(fse, 30, 1, "persistent"))


def test_no_loss_frame(fse, ctx):
    img = fse_synth.make_image(64, 96, 7)
    mask = np.zeros_like(img)
    p = _params(fse, 50, 1, "persistent")
    (out,), _ = gpu_conceal(ctx, [(img, mask)], p, want_work=False)
    assert np.array_equal(out, img)
    assert ctx.fse_last_batch_info()["lost_blocks"] == 0


def test_all_lost_frame(fse, ctx):
    img = fse_synth.make_image(64, 64, 8)
    mask = np.ones_like(img)
    for order in (0, 1):
        p = _params(fse, 40, order, "persistent")
        run_and_compare(ctx, [(img, mask)], p, "all lost")


def test_pixel_granular_mask(fse, ctx):
    """Losses that cover only parts of blocks (B_i smaller than the block)."""
    img = fse_synth.make_image(96, 96, 9)
    rng = np.random.default_rng(9)
    mask = (rng.random(img.shape) < 0.05).astype(np.uint8)
    mask[40:56, 10:30] = 1
    for order in (0, 1):
        p = _params(fse, 80, order, "persistent")
        run_and_compare(ctx, [(img, mask)], p, "pixel mask")


def test_isolated_losses_orders_identical(fse, ctx):
    img = fse_synth.make_image(128, 128, 21)
    lost = np.zeros((8, 8), np.uint8)
    lost[1::3, 1::3] = 1
    mask = fse_synth.blocks_to_pixel_mask(lost, 128, 128)
    r = []
    for order in (0, 1):
        p = _params(fse, 100, order, "persistent")
        outs, works = gpu_conceal(ctx, [(img, mask)], p)
        r.append((outs[0], works[0]))
    assert np.array_equal(r[0][0], r[1][0])
    assert np.array_equal(r[0][1], r[1][1], equal_nan=True)


def test_multi_frame_batch_matches_single(fse, ctx):
    frames = [fse_synth.random_frame(h, w, rate, s) for (h, w, rate, s) in
              [(80, 96, 0.3, 11), (128, 64, 0.5, 12), (48, 160, 0.2, 13)]]
    p = _params(fse, 80, 1, "persistent")
    outs, works, traces, _ = run_and_compare(ctx, frames, p, "batch")
    for i, (img, mask) in enumerate(frames):
        o1, w1 = gpu_conceal(ctx, [(img, mask)], p)
        assert np.array_equal(outs[i], o1[0])
        assert np.array_equal(works[i], w1[0], equal_nan=True)


def test_host_entry_point_matches_device(fse, ctx):
    img, mask = fse_synth.workload_mixed_512()[0]
    p = _params(fse, 100, 1, "persistent")
    (dev_out,), _ = gpu_conceal(ctx, [(img, mask)], p, want_work=False)
    out = np.empty_like(img)
    ctx.fse_conceal_batch_host([(img, mask, out)], p)
    assert np.array_equal(out, dev_out)


@pytest.mark.parametrize("h,w", [(37, 53), (100, 130), (64, 200)])
@pytest.mark.parametrize("executor", EXECS)
def test_host_entry_odd_sizes_pixel_losses(fse, ctx, h, w, executor):
    """Widths that are not a multiple of 16: device frames with such a row
    pitch are gathered with plain loads, while the host-frame path pads the
    device rows to 16 bytes and stages the areas with TMA; its block-loss maps
    come from the host masks.  Both must give the same bytes."""
    img = fse_synth.make_image(h, w, 500 + h + w)
    rng = np.random.default_rng(h * w)
    mask = (rng.random(img.shape) < 0.05).astype(np.uint8)
    mask[h // 4:h // 4 + 20, w // 3:w // 3 + 25] = 1
    p = _params(fse, 60, 1, executor)
    (dev_out,), _ = gpu_conceal(ctx, [(img, mask)], p, want_work=False)
    out = np.empty_like(img)
    ctx.fse_conceal_batch_host([(img, mask, out)], p)
    assert np.array_equal(out, dev_out)


def test_full_size_batch_sampled_frames(fse, ctx):
    """16 x 1920x1080, K = 200, one persistent launch (the benchmark's
    configuration); frames 0 and 5 are recomputed by the oracle in full."""
    frames = fse_synth.workload_batch_1080p(16)
    p = _params(fse, 200, 1, "persistent")
    *_, st = run_and_compare(ctx, frames, p, "1080p", sample=(0, 5))
    print(st)


@pytest.mark.parametrize("executor", EXECS)
def test_max_iterations(fse, ctx, executor):
    """K = FSE_MAX_ITERS, the largest K the C-ABI accepts: the (u, dc) list
    and the selection trace at their largest, against the oracle.  Every
    iteration is a chance of a near-tie that FP32 cannot resolve (late
    iterations pick among small, nearly equal residual energies), so more
    blocks have a near-tie in their FP64 trajectory than at K = 200; each
    root must be one of those, diverge at a near-tie and follow a valid
    trajectory."""
    img, mask = fse_synth.random_frame(64, 96, 0.35, 71)
    p = _params(fse, fse.FSE_MAX_ITERS, 1, executor)
    *_, st = run_and_compare(ctx, [(img, mask)], p, f"K={fse.FSE_MAX_ITERS}")
    print(st)


def test_uhd_frame(fse, ctx):
    """The largest frame of the serving mix, 3840x2160 (240 x 135 blocks),
    15% mixed isolated/burst losses plus a lost block-row slice, one
    persistent launch, recomputed in full by the oracle."""
    img = fse_synth.make_image(2160, 3840, 1077)
    rng = np.random.default_rng(2077)
    lost = fse_synth.mixed_block_mask(135, 240, 0.15, rng)
    lost = fse_synth.slice_rows(lost, 1, rng)
    mask = fse_synth.blocks_to_pixel_mask(lost, 2160, 3840)
    p = _params(fse, 200, 1, "persistent")
    *_, st = run_and_compare(ctx, [(img, mask)], p, "3840x2160")
    print(st)


# ---------------------------------------------------------------------------
# The per-block computation alone (pre-gathered areas)
# ---------------------------------------------------------------------------

def _random_areas(n, seed):
    rng = np.random.default_rng(seed)
    f = np.empty((n, 48, 48), np.float32)
    cls = np.zeros((n, 48, 48), np.uint8)
    for i in range(n):
        img = fse_synth.make_image(48, 48, 5000 + seed * 100 + i)
        f[i] = img
        cls[i, 16:32, 16:32] = oracle.CLS_BI
        kind = i % 5
        if kind == 1:
            cls[i, 0:16, :] = oracle.CLS_R
        elif kind == 2:
            cls[i, :, 32:48] = oracle.CLS_BO
            cls[i, 32:48, :] = oracle.CLS_R
        elif kind == 3:
            cls[i, 0:16, :] = oracle.CLS_OUT
            cls[i, :, 0:16] = oracle.CLS_OUT
        elif kind == 4:
            cls[i][rng.random((48, 48)) < 0.3] = oracle.CLS_BO
            cls[i, 16:32, 16:32] = oracle.CLS_BI
    return f, cls


@pytest.mark.parametrize("K", [1, 7, 100, 200, 1024])
def test_areas_against_oracle(fse, ctx, K):
    """Pre-gathered areas (all classes, image borders): traces equal to the
    oracle's give samples within 0.5; a trace that differs starts at one of
    the oracle's near-ties (margin within tau) and is a valid trajectory.
    The FP32 residual after the last update equals DFT{w (f - g)} of the
    GPU's own model within tau / 2 (tau = 2^-20 (sum|w f| + W[0] sum|dc|)):
    the measured error of the FP32 state that the validity bound assumes."""
    import torch
    n = 20
    f, cls = _random_areas(n, K)
    p = _params(fse, K, 1, "persistent")
    dev = torch.device("cuda:0")
    tf = torch.from_numpy(f).to(dev)
    tc = torch.from_numpy(cls).to(dev)
    g = torch.empty((n, 16, 16), dtype=torch.float32, device=dev)
    u = torch.empty((n, K), dtype=torch.int32, device=dev)
    dc = torch.empty((n, K, 2), dtype=torch.float32, device=dev)
    r = torch.empty((n, 64, 64, 2), dtype=torch.float32, device=dev)
    ctx.fse_extrapolate_areas(tf, tc, p, g, u, dc, r)
    torch.cuda.synchronize()
    g, u, dc, r = g.cpu().numpy(), u.cpu().numpy(), dc.cpu().numpy(), r.cpu().numpy()
    diverged = at_risk = 0
    worst_state = 0.0
    mm, nn = np.mgrid[0:48, 0:48]
    for i in range(n):
        f64 = f[i].astype(np.float64)
        ref = oracle.extrapolate_area(f64, cls[i], 64, K, 0.7, 0.2, 0.5)
        risky = bool((ref.margin <= TAU_SCALE).any())
        at_risk += risky
        if np.array_equal(u[i], ref.u):
            err = np.abs(g[i] - ref.g[16:32, 16:32]).max()
            assert err <= 0.5, (i, err)
        else:
            diverged += 1
            it, tie = near_tie_at_divergence(f64, cls[i], u[i], ref.u, 0.7, 0.2, 0.5)
            assert tie <= 1.0, (i, it, tie)
            assert ref.margin[it] <= TAU_SCALE, (i, it, ref.margin[it])
            worst, gv = trajectory(f64, cls[i], u[i], 0.7, 0.2, 0.5)
            assert worst <= 1.0 and np.abs(gv - g[i]).max() <= 0.5, (i, worst)
        # the GPU residual equals the spatial definition for its own trace
        d_gpu = dc[i, :, 0].astype(np.float64) + 1j * dc[i, :, 1]
        model = np.zeros((48, 48), complex)
        for uu, d in zip(u[i], d_gpu):
            model += d * np.exp(2j * np.pi * ((uu // 64) * mm + (uu % 64) * nn) / 64)
        x = np.zeros((64, 64), complex)
        x[:48, :48] = ref.w * (f64 - model)
        spatial = np.fft.fft2(x)
        rg = r[i, ..., 0] + 1j * r[i, ..., 1]
        scale = np.abs(ref.w * f64).sum() + ref.w.sum() * np.abs(d_gpu).sum()
        state = float(np.abs(rg - spatial).max() / scale)
        worst_state = max(worst_state, state)
        assert state <= TAU_SCALE / 2, (i, state / TAU_SCALE)
    print(f"K={K}: diverged {diverged}, at risk {at_risk}, "
          f"worst FP32 state error {worst_state / TAU_SCALE:.4f} tau")
    assert diverged <= at_risk


def test_area_without_support(fse, ctx):
    import torch
    dev = torch.device("cuda:0")
    f = torch.full((1, 48, 48), 100.0, device=dev)
    c = torch.full((1, 48, 48), oracle.CLS_BO, dtype=torch.uint8, device=dev)
    g = torch.empty((1, 16, 16), device=dev)
    u = torch.empty((1, 5), dtype=torch.int32, device=dev)
    ctx.fse_extrapolate_areas(f, c, _params(fse, 5, 1, "persistent"), g, u)
    torch.cuda.synchronize()
    assert torch.all(g == 0) and torch.all(u == -1)


# ---------------------------------------------------------------------------
# Errors and bounded waits
# ---------------------------------------------------------------------------

def test_invalid_params_rejected(fse, ctx):
    img, mask = fse_synth.workload_single_128()[0]
    out = np.empty_like(img)
    bad = [dict(iters=-1), dict(iters=fse.FSE_MAX_ITERS + 1), dict(rho=1.0), dict(rho=0.0),
           dict(delta=1.5), dict(gamma=0.0), dict(order=3), dict(executor=9),
           dict(block=3), dict(block=32), dict(border=8), dict(dft=32), dict(precision=42)]
    for kw in bad:
        p = fse.make_params(**{**dict(iters=10), **kw})
        with pytest.raises(fse.FseError) as e:
            ctx.fse_conceal_batch_host([(img, mask, out)], p)
        assert e.value.code == 1, kw


def test_device_wait_timeout_reports_status(fse, ctx):
    """A dependency that nothing releases makes the bounded device wait give
    up; the host sees FSE_ETIMEDOUT and the context stays usable."""
    img, mask = fse_synth.random_frame(64, 64, 0.5, 31)
    out = np.empty_like(img)
    p = _params(fse, 20, 1, "persistent")
    ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 2000)
    ctx.fse_ctx_set_option(fse.FSE_OPT_TEST_STUCK_DEP, 1)
    with pytest.raises(fse.FseError) as e:
        ctx.fse_conceal_batch_host([(img, mask, out)], p)
    assert e.value.code == 4
    ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 1 << 23)
    ctx.fse_conceal_batch_host([(img, mask, out)], p)
    (ref,), _ = gpu_conceal(ctx, [(img, mask)], p, want_work=False)
    assert np.array_equal(out, ref)


def test_autotune_same_bytes_and_cached(fse, ctx):
    """FSE_OPT_AUTOTUNE picks among launch configurations with identical
    results: the output equals the untuned one, the first call of a shape
    tunes, and the second reuses the choice."""
    frames = [fse_synth.random_frame(h, w, rate, s) for (h, w, rate, s) in
              [(96, 128, 0.3, 41), (64, 80, 0.5, 42)]]
    p = _params(fse, 60, 1, "persistent")
    ref_out, ref_work = gpu_conceal(ctx, frames, p)
    ctx.fse_ctx_set_option(fse.FSE_OPT_AUTOTUNE, 1)
    try:
        out1, work1 = gpu_conceal(ctx, frames, p)
        cfg1 = ctx.fse_last_batch_shape()
        out2, work2 = gpu_conceal(ctx, frames, p)
        cfg2 = ctx.fse_last_batch_shape()
    finally:
        ctx.fse_ctx_set_option(fse.FSE_OPT_AUTOTUNE, 0)
    for a, b in zip(ref_out + ref_work, out1 + work1):
        assert np.array_equal(a, b, equal_nan=True)
    for a, b in zip(ref_out + ref_work, out2 + work2):
        assert np.array_equal(a, b, equal_nan=True)
    assert cfg1 == cfg2
    if cfg1["executor"] == fse.FSE_EXEC_PERSISTENT:
        assert 1 <= cfg1["ctas_per_sm"] <= 3
        assert cfg1["claim_order"] in (fse.FSE_CLAIM_DELAYED, fse.FSE_CLAIM_HEIGHT,
                                       fse.FSE_CLAIM_LIST)
    else:
        assert cfg1["executor"] == fse.FSE_EXEC_GROUPS and cfg1["ctas_per_sm"] == 0
    assert cfg1["threads_per_cta"] == 256 and cfg1["blocks_per_cta"] == 1
    print(cfg1)


@pytest.mark.parametrize("claim", ["delayed", "height", "list"])
def test_claim_orders_same_bytes(fse, ctx, claim):
    """Every claim order of the persistent executor (the autotuner's third
    dimension) gives the bytes of the per-level launches: a block waits only
    for the earlier-group blocks in its area."""
    frames = [fse_synth.random_frame(h, w, rate, s) for (h, w, rate, s) in
              [(160, 224, 0.35, 43), (96, 96, 0.6, 44)]]
    ref_out, ref_work = gpu_conceal(ctx, frames, _params(fse, 80, 1, "groups"))
    mode = {"delayed": fse.FSE_CLAIM_DELAYED, "height": fse.FSE_CLAIM_HEIGHT,
            "list": fse.FSE_CLAIM_LIST}[claim]
    ctx.fse_ctx_set_option(fse.FSE_OPT_CLAIM_ORDER, mode)
    try:
        out, work = gpu_conceal(ctx, frames, _params(fse, 80, 1, "persistent"))
        assert ctx.fse_last_batch_shape()["claim_order"] == mode
    finally:
        ctx.fse_ctx_set_option(fse.FSE_OPT_CLAIM_ORDER, fse.FSE_CLAIM_DELAYED)
    for a, b in zip(ref_out + ref_work, out + work):
        assert np.array_equal(a, b, equal_nan=True)


def test_inputs_ready_pipelined_planning(fse, ctx):
    """FSE_OPT_INPUTS_READY: masks copied to the host on a side stream and
    batches planned while the previous one runs.  Back-to-back calls on
    different frames give the bytes of the default mode; a failed device
    wait is reported by a later call."""
    import torch
    dev = torch.device("cuda:0")
    sets = [[fse_synth.random_frame(h, w, rate, s)] for (h, w, rate, s) in
            [(96, 160, 0.3, 51), (128, 96, 0.45, 52), (64, 64, 0.6, 53)]]
    p = _params(fse, 60, 1, "persistent")
    ref = [gpu_conceal(ctx, fr, p, want_work=False)[0][0] for fr in sets]
    tens = [[(torch.from_numpy(i).to(dev), torch.from_numpy(m).to(dev),
              torch.empty_like(torch.from_numpy(i)).to(dev)) for i, m in fr] for fr in sets]
    ctx.fse_ctx_set_option(fse.FSE_OPT_INPUTS_READY, 1)
    try:
        for t in tens:  # no synchronisation between the calls
            ctx.fse_conceal_batch(t, p)
        torch.cuda.synchronize()
        for t, r in zip(tens, ref):
            assert np.array_equal(t[0][2].cpu().numpy(), r)
        ks = ctx.fse_recent_kernel_ms(3)
        assert len(ks) == 3 and all(k > 0 for k in ks)
        assert ks[0] == pytest.approx(ctx.fse_last_kernel_ms())
        # a dependency that nothing releases: the error surfaces later
        ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 2000)
        ctx.fse_ctx_set_option(fse.FSE_OPT_TEST_STUCK_DEP, 1)
        ctx.fse_conceal_batch(tens[0], p)
        torch.cuda.synchronize()
        with pytest.raises(fse.FseError) as e:
            ctx.fse_conceal_batch(tens[1], p)
        assert e.value.code == 4
        ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 1 << 23)
        ctx.fse_conceal_batch(tens[2], p)
        torch.cuda.synchronize()
        assert np.array_equal(tens[2][0][2].cpu().numpy(), ref[2])
    finally:
        ctx.fse_ctx_set_option(fse.FSE_OPT_INPUTS_READY, 0)
        ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 1 << 23)


def test_host_async_pipeline(fse, ctx):
    """fse_conceal_batch_host_async: three batches enqueued back to back
    (the third call waits for the first itself) give the bytes of the
    synchronous call; each ticket is waited for once; a failed device wait
    is reported by its own batch's wait and not by the next batch's."""
    import torch
    sets = [fse_synth.random_frame(h, w, rate, s) for (h, w, rate, s) in
            [(96, 160, 0.3, 61), (128, 96, 0.45, 62), (64, 64, 0.6, 63)]]
    p = _params(fse, 60, 1, "persistent")
    ref = []
    for img, mask in sets:
        out = np.empty_like(img)
        ctx.fse_conceal_batch_host([(img, mask, out)], p)
        ref.append(out)
    pinned = [(torch.from_numpy(i).pin_memory(), torch.from_numpy(m).pin_memory(),
               torch.zeros(i.shape, dtype=torch.uint8).pin_memory()) for i, m in sets]
    tickets = [ctx.fse_conceal_batch_host_async([b], p) for b in pinned]
    assert len(set(tickets)) == 3
    for t in reversed(tickets):
        ctx.fse_wait_batch(t)
    for (_, _, o), r in zip(pinned, ref):
        assert np.array_equal(o.numpy(), r)
    with pytest.raises(fse.FseError) as e:
        ctx.fse_wait_batch(tickets[0])
    assert e.value.code == 6  # FSE_ENOTFOUND
    # a dependency that nothing releases, in the first of two batches
    try:
        ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 2000)
        ctx.fse_ctx_set_option(fse.FSE_OPT_TEST_STUCK_DEP, 1)
        t_bad = ctx.fse_conceal_batch_host_async([pinned[0]], p)
        ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 1 << 23)
        t_ok = ctx.fse_conceal_batch_host_async([pinned[1]], p)
        ctx.fse_wait_batch(t_ok)
        with pytest.raises(fse.FseError) as e:
            ctx.fse_wait_batch(t_bad)
        assert e.value.code == 4  # FSE_ETIMEDOUT
        assert np.array_equal(pinned[1][2].numpy(), ref[1])
    finally:
        ctx.fse_ctx_set_option(fse.FSE_OPT_SPIN_LIMIT, 1 << 23)
        ctx.fse_ctx_set_option(fse.FSE_OPT_TEST_STUCK_DEP, 0)


def test_w_tables_change_no_byte(fse, ctx):
    """FSE_OPT_W_TABLES = 1: blocks whose sub-area classes follow from their
    eight neighbours take W from a per-pattern table computed once per
    context by the blocks' own FP32 split DFTs.  Outputs and FP32 working
    values are byte-identical to every block computing W itself, for the
    first call (tables filled) and a second one (tables reused), in both
    executors; frames with partial edge blocks and pixel-granular losses mix
    blocks with and without tables."""
    frames = fse_synth.workload_batch_1080p(2) + [fse_synth.random_frame(200, 264, 0.3, 91)]
    img, _ = fse_synth.workload_mixed_512()[0]
    rng = np.random.default_rng(92)
    pix = (rng.random(img.shape) < 0.02).astype(np.uint8)
    pix[100:164, 200:280] = 1
    frames.append((img, pix))
    for ex in ("persistent", "groups"):
        p = _params(fse, 200, 1, ex)
        ctx.fse_ctx_set_option(fse.FSE_OPT_W_TABLES, 0)
        try:
            ref_out, ref_work = gpu_conceal(ctx, frames, p)
            ctx.fse_ctx_set_option(fse.FSE_OPT_W_TABLES, 1)
            for _ in range(2):
                out, work = gpu_conceal(ctx, frames, p)
                for a, b in zip(ref_out + ref_work, out + work):
                    assert np.array_equal(a, b, equal_nan=True), ex
        finally:
            ctx.fse_ctx_set_option(fse.FSE_OPT_W_TABLES, 2)


def test_phase_clocks(fse, ctx):
    """FSE_OPT_PHASE_CLOCKS: the persistent executor records thread 0's SM
    clock at every phase boundary of every block; the outputs are those of
    the run without the stamps, and the iterations dominate at K = 200."""
    frames = fse_synth.workload_batch_1080p(1)
    p = _params(fse, 200, 1, "persistent")
    ref_out, ref_work = gpu_conceal(ctx, frames, p)
    ctx.fse_ctx_set_option(fse.FSE_OPT_PHASE_CLOCKS, 1)
    try:
        out, work = gpu_conceal(ctx, frames, p)
        clk, nb = ctx.fse_last_phase_clocks()
    finally:
        ctx.fse_ctx_set_option(fse.FSE_OPT_PHASE_CLOCKS, 0)
    for a, b in zip(ref_out + ref_work, out + work):
        assert np.array_equal(a, b, equal_nan=True)
    assert nb == ctx.fse_last_batch_info()["lost_blocks"]
    assert all(v >= 0 for v in clk.values())
    total = sum(clk.values())
    assert clk["iterations"] > 0.5 * total, clk
    print({k: round(v) for k, v in clk.items()})
