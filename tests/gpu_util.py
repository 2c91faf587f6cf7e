"""Helpers of the GPU parity tests: run frames through the C-ABI and compare
with the FP64 oracle.

Tolerance (floating point): every concealed sample's FP32 working value is
within 0.5 of the oracle's FP64 value on the 8-bit scale, and the PSNR of the
concealed samples against the oracle is at least 50 dB.  The 8-bit output is
checked in the kernel's own precision: out == round-half-even(FP32 value).
"""
from __future__ import annotations

import numpy as np

import oracle

TOL_ABS = 0.5
TOL_PSNR_DB = 50.0


def gpu_conceal(ctx, frames, params, want_work=True):
    """frames: list of (img uint8, mask uint8).  Returns lists of outputs
    (uint8) and FP32 working frames (NaN where not lost)."""
    import torch
    dev = torch.device("cuda:0")
    tens = []
    for img, mask in frames:
        l = torch.from_numpy(np.ascontiguousarray(img)).to(dev)
        m = torch.from_numpy(np.ascontiguousarray(mask)).to(dev)
        tens.append((l, m, torch.empty_like(l)))
    ctx.fse_conceal_batch(tens, params)
    outs, works = [], []
    for i, (l, m, o) in enumerate(tens):
        if want_work:
            wk = torch.empty(l.shape, dtype=torch.float32, device=dev)
            ctx.fse_copy_work(i, wk)
            torch.cuda.synchronize()
            w = wk.cpu().numpy().astype(np.float64)
            w[frames[i][1] == 0] = np.nan
            works.append(w)
        torch.cuda.synchronize()
        outs.append(o.cpu().numpy())
    return outs, works


def oracle_conceal(img, mask, params, threads=None):
    if threads is None:
        threads = oracle.max_threads()
    return oracle.conceal_frame(img, mask, block=params.block, border=params.border,
                                dft=params.dft, iters=params.iters, rho=params.rho,
                                delta=params.delta, gamma=params.gamma, order=params.order,
                                threads=threads)


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(255.0 ** 2 / mse)


def check_frame(img, mask, out, work, o_work, o_out, label=""):
    lost = mask != 0
    assert np.array_equal(out[~lost], img[~lost]), f"{label}: known samples changed"
    if lost.any():
        g = work[lost]
        r = o_work[lost]
        assert np.all(np.isfinite(g)), f"{label}: non-finite working values"
        err = np.abs(g - r)
        assert err.max() <= TOL_ABS, f"{label}: max |gpu - oracle| = {err.max():.4f}"
        assert psnr(g, r) >= TOL_PSNR_DB, f"{label}: PSNR {psnr(g, r):.2f} dB"
        # quantisation decided in the kernel's precision
        q = np.rint(work[lost].astype(np.float32)).astype(np.int64)
        assert np.array_equal(out[lost].astype(np.int64), q), f"{label}: out != rint(work)"
        return float(err.max()), psnr(g, r)
    return 0.0, float("inf")
