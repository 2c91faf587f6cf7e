"""Serving through fse_submit / fse_poll: continuous batching of requests of
different frame sizes and loss patterns; every result is the same alone and
in the mix, and sampled requests meet the parity criterion against the
oracle."""
import time

import numpy as np
import pytest

import fse_synth
from gpu_util import run_and_compare

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


def _requests(n, sizes=((288, 352), (720, 1280), (288, 352), (1080, 1920))):
    reqs = []
    for i in range(n):
        h, w = sizes[i % len(sizes)]
        img, mask = fse_synth.random_frame(h, w, 0.05 + 0.45 * ((i * 37) % 10) / 10.0, 700 + i)
        if i % 5 == 4:
            lost = np.zeros(fse_synth.block_grid(h, w), np.uint8)
            lost[2, :] = 1
            mask = np.maximum(mask, fse_synth.blocks_to_pixel_mask(lost, h, w))
        reqs.append((img, mask))
    return reqs


def test_results_same_alone_and_in_the_mix(fse):
    params = fse.make_params(iters=60, order=fse.FSE_ORDER_OPTIMIZED,
                             executor=fse.FSE_EXEC_PERSISTENT)
    reqs = _requests(10)
    with fse.Context(0) as ctx:
        alone = []
        for img, mask in reqs:
            out = np.empty_like(img)
            ctx.fse_conceal_batch_host([(img, mask, out)], params)
            alone.append(out)
        ctx.fse_ctx_set_option(fse.FSE_OPT_SERVE_SLOTS, 2)
        ctx.fse_ctx_set_option(fse.FSE_OPT_SERVE_MAX_BATCH, 4)
        outs = [np.full_like(img, 7) for img, _ in reqs]
        tickets = []
        # a burst: requests arrive while earlier batches are on the GPU
        for i, (img, mask) in enumerate(reqs):
            t = ctx.fse_submit(img, mask, outs[i], params)
            assert t > 0
            tickets.append(t)
        ctx.fse_drain(60000)
        stats = [ctx.fse_poll(t) for t in tickets]
        assert all(s is not None and s.status == 0 for s in stats)
        for i in range(len(reqs)):
            assert np.array_equal(outs[i], alone[i]), i
        assert max(s.batch_requests for s in stats) >= 2  # requests were batched
        assert max(s.inflight for s in stats) >= 1        # batches overlapped
        # and spaced arrivals: each is admitted as soon as a slot is free
        outs2 = [np.empty_like(img) for img, _ in reqs[:4]]
        t2 = []
        for i, (img, mask) in enumerate(reqs[:4]):
            t2.append(ctx.fse_submit(img, mask, outs2[i], params))
            time.sleep(0.003)
        ctx.fse_drain(60000)
        for i, t in enumerate(t2):
            assert ctx.fse_poll(t).status == 0
            assert np.array_equal(outs2[i], alone[i])
        for s, (img, mask) in zip(stats, reqs):
            assert s.lost_blocks == int(
                (np.add.reduceat(np.add.reduceat(mask, np.arange(0, mask.shape[0], 16), 0),
                                 np.arange(0, mask.shape[1], 16), 1) > 0).sum())
            assert s.latency_ms >= s.queue_ms >= 0
        with pytest.raises(fse.FseError):
            ctx.fse_poll(tickets[0])  # released after completion
    # Sampled requests against the oracle with the full parity criterion of
    # the batch path (sample by sample on clean blocks, validity elsewhere):
    # the batch path with traces gives the same bytes as the served result.
    with fse.Context(0) as tctx:
        tctx.fse_ctx_set_option(fse.FSE_OPT_KEEP_TRACE, 1)
        for i in (0, 3):
            dev_outs, _, _, st = run_and_compare(tctx, [reqs[i]], params, f"served request {i}")
            assert np.array_equal(outs[i], dev_outs[0]), i
            print(i, st)


def test_mixed_parameters_are_batched_separately(fse):
    reqs = _requests(4, sizes=((96, 128),))
    pa = fse.make_params(iters=30)
    pb = fse.make_params(iters=50, order=fse.FSE_ORDER_LINESCAN)
    with fse.Context(0) as ctx:
        ref = []
        for i, (img, mask) in enumerate(reqs):
            out = np.empty_like(img)
            ctx.fse_conceal_batch_host([(img, mask, out)], pa if i % 2 == 0 else pb)
            ref.append(out)
        outs = [np.empty_like(img) for img, _ in reqs]
        ts = [ctx.fse_submit(img, mask, outs[i], pa if i % 2 == 0 else pb)
              for i, (img, mask) in enumerate(reqs)]
        ctx.fse_drain(30000)
        for t in ts:
            assert ctx.fse_poll(t).status == 0
        for a, b in zip(outs, ref):
            assert np.array_equal(a, b)


def test_memory_budget_admission(fse):
    """A small budget serialises batches but every request completes; a
    request that can never fit fails with FSE_ENOMEM instead of waiting."""
    reqs = _requests(6, sizes=((288, 352),))
    params = fse.make_params(iters=20)
    with fse.Context(0, mem_budget=8 << 20) as ctx:
        outs = [np.empty_like(img) for img, _ in reqs]
        ts = [ctx.fse_submit(img, mask, outs[i], params) for i, (img, mask) in enumerate(reqs)]
        ctx.fse_drain(60000)
        st = [ctx.fse_poll(t) for t in ts]
        assert all(s.status == 0 for s in st)
        big, bmask = fse_synth.random_frame(2160, 3840, 0.2, 99)
        bout = np.empty_like(big)
        t = ctx.fse_submit(big, bmask, bout, params)
        ctx.fse_drain(60000)
        assert ctx.fse_poll(t).status == 2


def test_page_locked_requests(fse):
    """Requests whose buffers are page-locked are copied without staging;
    mixed in one batch with pageable ones, every result equals the
    synchronous call's."""
    import torch
    params = fse.make_params(iters=60, order=fse.FSE_ORDER_OPTIMIZED,
                             executor=fse.FSE_EXEC_PERSISTENT)
    reqs = _requests(6)
    with fse.Context(0) as ctx:
        alone = []
        for img, mask in reqs:
            out = np.empty_like(img)
            ctx.fse_conceal_batch_host([(img, mask, out)], params)
            alone.append(out)
        keep, bufs = [], []
        for i, (img, mask) in enumerate(reqs):
            if i % 2 == 0:  # page-locked: numpy views of pinned tensors
                t = [torch.from_numpy(a).pin_memory() for a in (img, mask)]
                t.append(torch.full(img.shape, 7, dtype=torch.uint8).pin_memory())
                keep.append(t)
                bufs.append(tuple(x.numpy() for x in t))
            else:
                bufs.append((img, mask, np.full_like(img, 7)))
        tickets = [ctx.fse_submit(l, m, o, params) for l, m, o in bufs]
        assert all(t > 0 for t in tickets)
        ctx.fse_drain(60000)
        for t, (_, _, o), ref in zip(tickets, bufs, alone):
            assert ctx.fse_poll(t).status == 0
            assert np.array_equal(o, ref)


def _offered_load(fse, ctx, params, reqs, seconds, interval_s):
    """Submit `reqs` cyclically every interval_s for `seconds`; returns
    (refused, [stats of completed requests])."""
    outs = [np.empty_like(img) for img, _ in reqs]
    tickets, refused = [], 0
    t0 = time.perf_counter()
    i = 0
    while time.perf_counter() - t0 < seconds:
        img, mask = reqs[i % len(reqs)]
        # each in-flight request needs its own output buffer
        out = outs[i % len(reqs)] if i < len(reqs) else np.empty_like(img)
        t = ctx.fse_submit(img, mask, out, params)
        if t < 0:
            refused += 1
        else:
            tickets.append((t, out))
        i += 1
        time.sleep(interval_s)
    ctx.fse_drain(120000)
    return refused, [ctx.fse_poll(t) for t, _ in tickets]


def test_latency_aware_admission(fse):
    """Offered load far above what the GPU sustains: without a latency
    budget every request is queued and the queueing delay grows with the
    backlog; with FSE_OPT_SERVE_LATENCY_MS = 20 requests are refused while
    the oldest queued one has waited longer than 20 ms, so the delays of the
    admitted requests stay bounded."""
    params = fse.make_params(iters=200, order=fse.FSE_ORDER_OPTIMIZED,
                             executor=fse.FSE_EXEC_PERSISTENT)
    reqs = [fse_synth.random_frame(1080, 1920, 0.5, 800 + i) for i in range(4)]
    res = {}
    for budget in (0, 20):
        with fse.Context(0) as ctx:
            ctx.fse_ctx_set_option(fse.FSE_OPT_SERVE_LATENCY_MS, budget)
            refused, stats = _offered_load(fse, ctx, params, reqs, 0.6, 0.0005)
        assert all(s is not None and s.status == 0 for s in stats)
        q = np.array([s.queue_ms for s in stats])
        res[budget] = (refused, len(stats), float(np.percentile(q, 90)), float(q.max()))
    print(res)
    assert res[0][0] == 0            # no budget: nothing refused ...
    assert res[20][0] > 0            # ... with a budget, the overload is refused
    assert res[20][2] < res[0][2]    # and the queueing delay is shorter
    assert res[20][3] <= 20.0 + 1000.0 * 0.6 / 4  # bounded: far below the unbounded backlog
