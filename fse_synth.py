"""Seeded synthetic inputs for FSE block-loss concealment.

The paper evaluates on the test images "Lena", "Peppers" and "Baboon" with
isolated, consecutive and mixed 16x16 loss patterns (Sec. 4, Fig. 3).  Those
images are not available, so this module generates stand-ins with the same
character: smooth oriented texture (sinusoids), step edges (filled polygons)
and sensor noise, in 8-bit luma, plus whole-block loss masks.

This module holds input generation only.  It contains none of the
extrapolation arithmetic and is shared by the CPU oracle tests, the GPU
parity tests and the benchmark.

Recipe (all draws from ``numpy.random.Generator(PCG64(seed))``):

* image: base value 128, plus 6 sinusoids with amplitude U(10, 60),
  orientation U(0, pi), period U(8, 64) px and phase U(0, 2 pi); then 3 filled
  polygons with 3-6 vertices uniform over the frame, each replacing the pixels
  it covers with a value U(0, 255); then Gaussian noise sigma = 2; rounded
  half-to-even and clipped to [0, 255].
* masks: whole 16x16 blocks (partial blocks at the right/bottom edge cover
  only their in-image pixels); a pixel value 1 marks a lost sample.
"""
from __future__ import annotations

import numpy as np

BLOCK = 16


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _fill_polygon(img: np.ndarray, xs: np.ndarray, ys: np.ndarray, value: float) -> None:
    """Even-odd rule fill, evaluated at pixel centres."""
    h, w = img.shape
    py, px = np.mgrid[0:h, 0:w].astype(np.float64)
    py += 0.5
    px += 0.5
    inside = np.zeros((h, w), dtype=bool)
    nv = len(xs)
    for i in range(nv):
        x0, y0 = xs[i], ys[i]
        x1, y1 = xs[(i + 1) % nv], ys[(i + 1) % nv]
        if y0 == y1:
            continue
        crosses = (y0 > py) != (y1 > py)
        xint = x0 + (py - y0) * (x1 - x0) / (y1 - y0)
        inside ^= crosses & (px < xint)
    img[inside] = value


def make_image(height: int, width: int, seed: int) -> np.ndarray:
    """Synthetic 8-bit luma frame (uint8, shape [height, width])."""
    rng = _rng(seed)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    img = np.full((height, width), 128.0)
    for _ in range(6):
        amp = rng.uniform(10.0, 60.0)
        theta = rng.uniform(0.0, np.pi)
        period = rng.uniform(8.0, 64.0)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        proj = xx * np.cos(theta) + yy * np.sin(theta)
        img += amp * np.sin(2.0 * np.pi * proj / period + phase)
    for _ in range(3):
        nv = int(rng.integers(3, 7))
        xs = rng.uniform(0.0, width, nv)
        ys = rng.uniform(0.0, height, nv)
        val = rng.uniform(0.0, 255.0)
        _fill_polygon(img, xs, ys, val)
    img += rng.normal(0.0, 2.0, size=img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def block_grid(height: int, width: int, block: int = BLOCK) -> tuple[int, int]:
    """(rows, cols) of the block grid; partial blocks count."""
    return (height + block - 1) // block, (width + block - 1) // block


def blocks_to_pixel_mask(lost_blocks: np.ndarray, height: int, width: int,
                         block: int = BLOCK) -> np.ndarray:
    """Expand a [BH, BW] block-loss map into a [H, W] uint8 pixel mask."""
    full = np.kron(lost_blocks.astype(np.uint8), np.ones((block, block), np.uint8))
    return np.ascontiguousarray(full[:height, :width])


def iid_block_mask(bh: int, bw: int, rate: float, rng: np.random.Generator) -> np.ndarray:
    """Each block lost independently with probability ``rate``."""
    return (rng.random((bh, bw)) < rate).astype(np.uint8)


def mixed_block_mask(bh: int, bw: int, rate: float, rng: np.random.Generator,
                     burst_len: tuple[int, int] = (4, 8)) -> np.ndarray:
    """Half of the target loss as horizontal bursts, the rest isolated blocks.

    Bursts of U{4..8} consecutive blocks in one block row are placed at random
    positions until half the target count is reached.  The remaining losses
    are single blocks whose 8-neighbours are all intact where such a block
    exists, otherwise any intact block.
    """
    lost = np.zeros((bh, bw), np.uint8)
    target = int(round(rate * bh * bw))
    half = target // 2
    lo, hi = burst_len
    while int(lost.sum()) < half:
        length = int(rng.integers(lo, hi + 1))
        length = min(length, bw)
        r = int(rng.integers(0, bh))
        c = int(rng.integers(0, bw - length + 1))
        lost[r, c:c + length] = 1
    while int(lost.sum()) < target:
        padded = np.pad(lost, 1)
        near = np.zeros_like(lost)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                near |= padded[1 + dy:1 + dy + bh, 1 + dx:1 + dx + bw]
        cand = np.flatnonzero(near.ravel() == 0)
        if cand.size == 0:
            cand = np.flatnonzero(lost.ravel() == 0)
        pick = int(cand[int(rng.integers(0, cand.size))])
        lost.ravel()[pick] = 1
    return lost


def slice_rows(lost: np.ndarray, count: int, rng: np.random.Generator) -> np.ndarray:
    """Add ``count`` consecutive full block-row slice losses."""
    bh = lost.shape[0]
    count = min(count, bh)
    r0 = int(rng.integers(0, bh - count + 1))
    out = lost.copy()
    out[r0:r0 + count, :] = 1
    return out


# ---------------------------------------------------------------------------
# Workloads.  Each returns a list of (image uint8 [H,W], pixel mask uint8 [H,W]).
# Image seed = 1000 + frame index, mask seed = 2000 + frame index.
# ---------------------------------------------------------------------------

def workload_single_128(frame: int = 0):
    """128x128 frame, 10% of 16x16 blocks lost i.i.d. (line-scan workload)."""
    h = w = 128
    img = make_image(h, w, 1000 + frame)
    bh, bw = block_grid(h, w)
    lost = iid_block_mask(bh, bw, 0.10, _rng(2000 + frame))
    return [(img, blocks_to_pixel_mask(lost, h, w))]


def workload_mixed_512(frame: int = 0):
    """512x512 frame, 25% of blocks lost: half bursts of 4-8 blocks, half isolated."""
    h = w = 512
    img = make_image(h, w, 1000 + frame)
    bh, bw = block_grid(h, w)
    lost = mixed_block_mask(bh, bw, 0.25, _rng(2000 + frame))
    return [(img, blocks_to_pixel_mask(lost, h, w))]


def workload_batch_1080p(frames: int = 16, height: int = 1080, width: int = 1920):
    """``frames`` 1920x1080 frames, each with its own i.i.d. loss rate U(5%, 50%)."""
    out = []
    bh, bw = block_grid(height, width)
    for f in range(frames):
        img = make_image(height, width, 1000 + f)
        rng = _rng(2000 + f)
        rate = rng.uniform(0.05, 0.50)
        lost = iid_block_mask(bh, bw, rate, rng)
        out.append((img, blocks_to_pixel_mask(lost, height, width)))
    return out


SERVING_SIZES = ((288, 352), (720, 1280), (1080, 1920), (2160, 3840))


def serving_request(index: int):
    """One request of the serving stream: size uniform over four formats,
    loss rate U(5%, 50%), and with probability 0.2 one or two extra full
    block-row slices."""
    rng = _rng(2000 + index)
    h, w = SERVING_SIZES[int(rng.integers(0, len(SERVING_SIZES)))]
    img = make_image(h, w, 1000 + index)
    bh, bw = block_grid(h, w)
    rate = rng.uniform(0.05, 0.50)
    lost = iid_block_mask(bh, bw, rate, rng)
    if rng.random() < 0.2:
        lost = slice_rows(lost, int(rng.integers(1, 3)), rng)
    return img, blocks_to_pixel_mask(lost, h, w)


def serving_image(fmt: int, variant: int):
    """Content of the serving stream: two images per format."""
    h, w = SERVING_SIZES[fmt]
    return make_image(h, w, 5000 + 10 * fmt + variant)


def serving_mask(index: int):
    """Format and loss mask of serving request `index` (the same draws as
    serving_request): size uniform over four formats, loss rate U(5%, 50%),
    with probability 0.2 one or two extra full block-row slices."""
    rng = _rng(2000 + index)
    fmt = int(rng.integers(0, len(SERVING_SIZES)))
    h, w = SERVING_SIZES[fmt]
    bh, bw = block_grid(h, w)
    rate = rng.uniform(0.05, 0.50)
    lost = iid_block_mask(bh, bw, rate, rng)
    if rng.random() < 0.2:
        lost = slice_rows(lost, int(rng.integers(1, 3)), rng)
    return fmt, blocks_to_pixel_mask(lost, h, w)


def random_frame(height: int, width: int, rate: float, seed: int):
    """Generic seeded frame + i.i.d. block mask for tests of arbitrary size."""
    img = make_image(height, width, 1000 + seed)
    bh, bw = block_grid(height, width)
    lost = iid_block_mask(bh, bw, rate, _rng(2000 + seed))
    return img, blocks_to_pixel_mask(lost, height, width)
