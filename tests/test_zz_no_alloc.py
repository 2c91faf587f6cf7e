"""fse_conceal_frame_noalloc: the allocation-free entry point for callers that
cannot call cudaMalloc (device memory owned by a host application's pool or
budget).  Its scratch is one fixed device array inside the library; the test
calls it through the C-ABI twice in a row, on two different frames, and
checks each result against the regular entry point fse_conceal_batch run
with the same parameters (groups executor, FP32), within the pixel
tolerance of the parity tests, in both processing orders.  It also covers a
frame concealed in place (out == luma) whose sides are not multiples of 16,
and the size limit.

Collected last on purpose: a run that stops at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import fse_synth

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


def _noalloc(fse, luma, mask, out, params, stream):
    h, w = luma.shape
    fr = fse.fse_frame(luma.data_ptr(), out.data_ptr(), mask.data_ptr(), w, h, luma.stride(0))
    return fse.lib().fse_conceal_frame_noalloc(ctypes.byref(fr), ctypes.byref(params), stream)


@pytest.mark.parametrize("order", ["optimized", "linescan"])
def test_noalloc_matches_regular_entry_point_twice(fse, order):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    optimized = order == "optimized"
    params = fse.make_params(iters=200 if optimized else 60, rho=0.7, delta=0.2, gamma=0.5,
                             order=fse.FSE_ORDER_OPTIMIZED if optimized else fse.FSE_ORDER_LINESCAN,
                             executor=fse.FSE_EXEC_GROUPS)
    if optimized:
        frames = [fse_synth.workload_mixed_512()[0],            # 512 x 512, mixed losses
                  fse_synth.random_frame(1080, 1920, 0.3, 41)]  # the size limit's frame
    else:  # line scan: one launch per lost block, so smaller frames
        frames = [fse_synth.workload_single_128()[0],
                  fse_synth.random_frame(200, 264, 0.3, 43)]
    tens = []
    for img, mask in frames:
        luma = torch.from_numpy(img).to(dev)
        m = torch.from_numpy(mask).to(dev)
        tens.append((luma, m, torch.zeros_like(luma), torch.zeros_like(luma)))
    # two calls in a row on the shared scratch
    for luma, m, out_na, _ in tens:
        rc = _noalloc(fse, luma, m, out_na, params, stream)
        assert rc == 0, fse.strerror(rc)
    torch.cuda.synchronize()
    with fse.Context(0) as ctx:
        # weight spectra by the blocks' own FP32 arithmetic, as this entry
        # point computes them (the default tensor-core tables round apart)
        ctx.fse_ctx_set_option(fse.FSE_OPT_W_TABLES, 1)
        for (img, mask), (luma, m, out_na, out_ref) in zip(frames, tens):
            ctx.fse_conceal_batch([(luma, m, out_ref)], params)
            torch.cuda.synchronize()
            a = out_na.cpu().numpy().astype(np.int32)
            b = out_ref.cpu().numpy().astype(np.int32)
            assert np.array_equal(a[mask == 0], img[mask == 0])
            assert np.abs(a - b).max() <= 1
            assert (a != b).sum() == 0


def test_noalloc_in_place_odd_size(fse):
    """out == luma (the lost samples are overwritten in place) on a frame of
    1080 x 1918 samples: partial blocks on the right edge, and a row pitch
    that is not a multiple of 16."""
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    params = fse.make_params(iters=100, order=fse.FSE_ORDER_OPTIMIZED,
                             executor=fse.FSE_EXEC_GROUPS)
    img, mask = fse_synth.random_frame(1080, 1918, 0.25, 44)
    buf = torch.from_numpy(img).to(dev)
    m = torch.from_numpy(mask).to(dev)
    for _ in range(2):  # the second call conceals an already concealed frame
        buf.copy_(torch.from_numpy(img))
        rc = _noalloc(fse, buf, m, buf, params, stream)
        assert rc == 0, fse.strerror(rc)
    torch.cuda.synchronize()
    got = buf.cpu().numpy()
    ref = np.empty_like(img)
    with fse.Context(0) as ctx:
        ctx.fse_ctx_set_option(fse.FSE_OPT_W_TABLES, 1)
        ctx.fse_conceal_batch_host([(img, mask, ref)], params)
    assert np.array_equal(got, ref)


def test_noalloc_rejects_frames_beyond_its_scratch(fse):
    import torch
    dev = torch.device("cuda:0")
    img, mask = fse_synth.random_frame(1088 + 16, 64, 0.2, 42)
    luma = torch.from_numpy(img).to(dev)
    m = torch.from_numpy(mask).to(dev)
    out = torch.empty_like(luma)
    rc = _noalloc(fse, luma, m, out, fse.make_params(iters=10), torch.cuda.current_stream().cuda_stream)
    assert rc == fse._native.FSE_ETOOBIG
    assert "1920 x 1088" in fse.strerror(rc)
