"""Block sizes 8, 4 and 2 with a 16-sample frame (Sec. 4 evaluates all four
block sizes).  The area (B + 32)^2 then reaches blocks beyond the
8-neighbourhood; blocks of one group read the frame as of the group start,
and the persistent executor must wait for every earlier-group block whose
samples lie in the area.  Checked against the FP64 oracle (both orders) and
by bit-identity of the two executors."""
import numpy as np
import pytest

import fse_synth
from gpu_util import gpu_conceal, run_and_compare

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


def _mixed(h, w, seed):
    """Whole 16x16 losses (isolated and in bursts), as in the paper's test
    patterns, to be concealed with smaller blocks."""
    img = fse_synth.make_image(h, w, 3000 + seed)
    rng = np.random.default_rng(seed)
    lost16 = fse_synth.mixed_block_mask((h + 15) // 16, (w + 15) // 16, 0.25, rng)
    return img, fse_synth.blocks_to_pixel_mask(lost16, h, w)


@pytest.mark.parametrize("B", [8, 4, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_small_blocks_against_oracle(fse, ctx, B, order):
    frames = [_mixed(80, 96, B)]
    p = fse.make_params(iters=60, order=order, block=B, executor=fse.FSE_EXEC_PERSISTENT)
    *_, st = run_and_compare(ctx, frames, p, f"B={B} order={order}")
    print(B, order, st)


@pytest.mark.parametrize("B", [8, 4, 2])
def test_small_blocks_executors_bit_identical(fse, ctx, B):
    img, mask = _mixed(128, 160, 10 + B)
    res = []
    for ex in (fse.FSE_EXEC_GROUPS, fse.FSE_EXEC_PERSISTENT):
        p = fse.make_params(iters=80, order=fse.FSE_ORDER_OPTIMIZED, block=B, executor=ex)
        outs, works = gpu_conceal(ctx, [(img, mask)], p)
        res.append((outs[0], works[0]))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1], equal_nan=True)


def test_small_blocks_partial_edges_and_pixel_losses(fse, ctx):
    img = fse_synth.make_image(37, 53, 77)
    rng = np.random.default_rng(77)
    mask = (rng.random(img.shape) < 0.08).astype(np.uint8)
    mask[10:20, 5:30] = 1
    for B in (8, 4, 2):
        p = fse.make_params(iters=40, order=fse.FSE_ORDER_OPTIMIZED, block=B)
        run_and_compare(ctx, [(img, mask)], p, f"edges B={B}")


def test_block_size_rejected_when_unsupported(fse, ctx):
    img, mask = _mixed(32, 32, 1)
    out = np.empty_like(img)
    for B in (1, 3, 32):
        with pytest.raises(fse.FseError):
            ctx.fse_conceal_batch_host([(img, mask, out)], fse.make_params(iters=5, block=B))
