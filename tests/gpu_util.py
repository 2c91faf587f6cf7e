"""Helpers of the GPU parity tests: run frames through the C-ABI and compare
with the FP64 oracle.

Tolerance (floating point): every concealed sample's FP32 working value is
within 0.5 of the oracle's FP64 value on the 8-bit scale, and the PSNR of the
concealed samples against the oracle is at least 50 dB.  The 8-bit output is
checked in the kernel's own precision: out == round-half-even(FP32 value).

The argmax of every iteration is a decision taken in floating point.  Where
the FP32 and FP64 energies of two candidates are closer than FP32 can
resolve, the two sides may pick different members of the near-tie, and from
there on (in that block and in blocks that read it as reconstructed area)
the extrapolated values are not unique.  Such blocks are checked for
validity (fse_check): the divergence starts at a near-tie of the oracle's
own trajectory, and the GPU result is a correct FSE trajectory on the
samples it saw.  All other blocks are compared with the oracle sample by
sample.

How many blocks may diverge is predicted by the oracle itself: a block can
only leave the oracle's trajectory at an iteration where the FP64 choice
wins by less than tau (its selection margin, fse_oracle.h).  Every root
(a diverged block whose earlier-group neighbours are all clean) must be such
an "at risk" block of the oracle's frame.
"""
from __future__ import annotations

import numpy as np

import oracle
from fse_check import area_from_frame, near_tie_at_divergence, tau_scale, trajectory

TOL_ABS = 0.5
TOL_PSNR_DB = 50.0


def gpu_conceal(ctx, frames, params, want_work=True, want_trace=False):
    """frames: list of (img uint8, mask uint8).  Returns lists of outputs
    (uint8), FP32 working frames (NaN where not lost) and, if asked, the
    selection traces [BH*BW, K] int16."""
    import torch
    dev = torch.device("cuda:0")
    tens = []
    for img, mask in frames:
        l = torch.from_numpy(np.ascontiguousarray(img)).to(dev)
        m = torch.from_numpy(np.ascontiguousarray(mask)).to(dev)
        tens.append((l, m, torch.empty_like(l)))
    ctx.fse_conceal_batch(tens, params)
    outs, works, traces = [], [], []
    for i, (l, m, o) in enumerate(tens):
        if want_work:
            wk = torch.empty(l.shape, dtype=torch.float32, device=dev)
            ctx.fse_copy_work(i, wk)
            torch.cuda.synchronize()
            w = wk.cpu().numpy().astype(np.float64)
            w[frames[i][1] == 0] = np.nan
            works.append(w)
        if want_trace:
            h, wd = l.shape
            B = params.block
            nb = ((h + B - 1) // B) * ((wd + B - 1) // B)
            t = torch.empty(nb * max(params.iters, 1), dtype=torch.int16, device=dev)
            ctx.fse_copy_trace(i, t)
            torch.cuda.synchronize()
            traces.append(t.cpu().numpy().astype(np.int32).reshape(nb, -1)[:, :params.iters])
        torch.cuda.synchronize()
        outs.append(o.cpu().numpy())
    if want_trace:
        return outs, works, traces
    return outs, works


def oracle_conceal(img, mask, params, threads=None, trace=False, margins=False):
    if threads is None:
        threads = oracle.max_threads()
    return oracle.conceal_frame(img, mask, block=params.block, border=params.border,
                                dft=params.dft, iters=params.iters, rho=params.rho,
                                delta=params.delta, gamma=params.gamma, order=params.order,
                                threads=threads, trace=trace, margins=margins)


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(255.0 ** 2 / mse)


def check_output_basics(img, mask, out, work, label=""):
    lost = mask != 0
    assert np.array_equal(out[~lost], img[~lost]), f"{label}: known samples changed"
    if lost.any():
        assert np.all(np.isfinite(work[lost])), f"{label}: non-finite working values"
        assert np.all((work[lost] >= 0) & (work[lost] <= 255))
        q = np.rint(work[lost].astype(np.float32)).astype(np.int64)
        assert np.array_equal(out[lost].astype(np.int64), q), f"{label}: out != rint(work)"


def compare_frame(img, mask, params, out, work, g_trace, o_work, o_trace, gob, label="",
                  o_margin=None):
    """Sample-by-sample parity on blocks whose selections and inputs agree
    with the oracle; validity on the others.  o_margin: the oracle's
    selection margins [BH*BW, K]; with them every root must be a block at
    risk.  Returns a statistics dict."""
    check_output_basics(img, mask, out, work, label)
    bh, bw = gob.shape
    B, d = params.block, params.border
    tau_s = tau_scale(params.precision)
    rad = d // B                     # blocks whose samples are in the area
    lost_blocks = [(int(gob[by, bx]), by, bx) for by in range(bh) for bx in range(bw)
                   if gob[by, bx] >= 0]
    lost_blocks.sort()
    clean = np.zeros((bh, bw), bool)
    at_risk = None
    if o_margin is not None:
        at_risk = (np.asarray(o_margin) <= tau_s).any(axis=1).reshape(bh, bw) & (gob >= 0)
    stats = dict(blocks=len(lost_blocks), clean=0, roots=0, downstream=0,
                 at_risk=None if at_risk is None else int(at_risk.sum()),
                 max_err_clean=0.0, worst_tie=0.0, worst_valid=0.0, max_err_valid=0.0)
    errs = []
    errs_all = []
    for g, by, bx in lost_blocks:
        b = by * bw + bx
        same = np.array_equal(g_trace[b], o_trace[b])
        up_clean = True
        for dy in range(-rad, rad + 1):
            for dx in range(-rad, rad + 1):
                ny, nx = by + dy, bx + dx
                if (dy or dx) and 0 <= ny < bh and 0 <= nx < bw:
                    if 0 <= gob[ny, nx] < g and not clean[ny, nx]:
                        up_clean = False
        ys = slice(by * B, min(by * B + B, img.shape[0]))
        xs = slice(bx * B, min(bx * B + B, img.shape[1]))
        lm = mask[ys, xs] != 0
        errs_all.append((work[ys, xs][lm], o_work[ys, xs][lm]))
        if same and up_clean:
            clean[by, bx] = True
            stats["clean"] += 1
            e = np.abs(work[ys, xs][lm] - o_work[ys, xs][lm])
            errs.append((work[ys, xs][lm], o_work[ys, xs][lm]))
            stats["max_err_clean"] = max(stats["max_err_clean"], float(e.max()))
            continue
        # not unique: the GPU result must be a valid trajectory on its inputs
        f, cls = area_from_frame(img, mask, work, gob, by, bx, B, d)
        worst, gv = trajectory(f, cls, g_trace[b], params.rho, params.delta, params.gamma,
                               B=B, d=d, tau_s=tau_s)
        assert worst <= 1.0, f"{label}: block ({by},{bx}) selection off by {worst:.2f} tau"
        gi = np.clip(gv, 0, 255)[:lm.shape[0], :lm.shape[1]]
        ev = float(np.abs(gi[lm] - work[ys, xs][lm]).max())
        assert ev <= TOL_ABS, f"{label}: block ({by},{bx}) model differs from its trajectory by {ev}"
        stats["worst_valid"] = max(stats["worst_valid"], worst)
        stats["max_err_valid"] = max(stats["max_err_valid"], ev)
        if up_clean:
            stats["roots"] += 1
            fo, clso = area_from_frame(img, mask, o_work, gob, by, bx, B, d)
            it, tie = near_tie_at_divergence(fo, clso, g_trace[b], o_trace[b], params.rho,
                                             params.delta, params.gamma, tau_s=tau_s)
            assert tie <= 1.0, f"{label}: block ({by},{bx}) diverged at it {it} by {tie:.2f} tau"
            stats["worst_tie"] = max(stats["worst_tie"], tie)
            if at_risk is not None:
                assert at_risk[by, bx], (
                    f"{label}: block ({by},{bx}) diverged but the oracle's trajectory has no "
                    f"near-tie within tau")
        else:
            stats["downstream"] += 1
    assert stats["max_err_clean"] <= TOL_ABS, f"{label}: {stats}"
    if errs:
        a = np.concatenate([x for x, _ in errs])
        r = np.concatenate([y for _, y in errs])
        stats["psnr_clean"] = psnr(a, r)
        assert stats["psnr_clean"] >= TOL_PSNR_DB, f"{label}: {stats}"
    if errs_all:
        a = np.concatenate([x for x, _ in errs_all])
        r = np.concatenate([y for _, y in errs_all])
        stats["max_err_all"] = float(np.abs(a - r).max())
        stats["psnr_all"] = psnr(a, r)
    if stats["blocks"]:
        stats["diverged_frac"] = 1.0 - stats["clean"] / stats["blocks"]
        stats["clean_frac"] = stats["clean"] / stats["blocks"]
        if at_risk is not None:
            # each root is an at-risk block (checked above), so their count
            # is bounded by the oracle's own near-ties
            assert stats["roots"] <= stats["at_risk"], f"{label}: {stats}"
    return stats


def run_and_compare(ctx, frames, params, label="", sample=None):
    """GPU batch with traces, oracle per (sampled) frame, compare_frame."""
    outs, works, traces = gpu_conceal(ctx, frames, params, want_trace=True)
    all_stats = []
    for i in (range(len(frames)) if sample is None else sample):
        img, mask = frames[i]
        o_work, o_out, gob, o_trace, o_margin = oracle_conceal(img, mask, params, trace=True,
                                                               margins=True)
        st = compare_frame(img, mask, params, outs[i], works[i], traces[i], o_work, o_trace, gob,
                           f"{label} frame {i}", o_margin)
        all_stats.append(st)
    return outs, works, traces, all_stats
