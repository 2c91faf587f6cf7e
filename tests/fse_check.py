"""FP64 validity check of a selection trajectory (Sec. 4 iteration).

The FP32 GPU path and the FP64 oracle take the same argmax decisions except
at near-ties, where the two precisions may pick different members of the
tie.  FSE's extrapolation into the lost area depends on which basis
function is picked, so from such a point on the result is not unique.  For
those blocks the tests check validity instead of equality: given the area
the GPU saw and the indices it selected, the weighted residual spectrum is
recomputed here in FP64 from the definitions (numpy FFT of the zero-extended
weighted area, transform-domain update) along the GPU's trajectory, and

* every selected index must maximise |R_w| within the error bound
  tau = s * (sum |w f| + W[0] * sum_i |dc_i|) of the GPU's spectrum: the
  first term scales the rounding of the projection (every entry of R_w is a
  weighted sum of the samples w f, so its error is a multiple of the unit
  roundoff times sum |w f|), the second the rounding of the residual updates
  (iteration i subtracts dc_i W[k - u_i], |W[k]| <= W[0]);
* the model built along the trajectory must reproduce the GPU's inserted
  samples within the pixel tolerance.

The factor s depends on the projection's arithmetic.  FP32 (and split TF32,
about 21 significant bits): s = 2^-20 = 16 u with u = 2^-24.  The split
row and column DFTs take every entry through 28 rounded additions and four
twiddle products; with independent roundings the error grows like
sqrt(28) u ~ 5 u, and the worst case of the first-order bound is ~36 u.  The
GPU tests measure the FP32 spectrum's error along the GPU's own trajectory
directly and require it to stay below tau / 2, so that a deficit of at most
tau (twice the state error) follows.  Split BF16 keeps about 16 significant
bits per operand (hi + lo, both 8-bit significands): s = 2^-16.
"""
from __future__ import annotations

import numpy as np

import oracle

TAU_SCALE = 2.0 ** -20          # FP32 projection (and split TF32)
TAU_SCALE_BY_PRECISION = {0: 2.0 ** -20, 5: 2.0 ** -20, 4: 2.0 ** -16}


def tau_scale(precision: int) -> float:
    """The factor s of tau for an FSE_PREC_* projection (FP32-grade ones
    only; single-pass TF32, BF16 and FP16 are not checked this way)."""
    return TAU_SCALE_BY_PRECISION[int(precision)]


def area_from_frame(img, mask, work, gob, by, bx, B=16, d=16):
    """The 48x48 area of block (by, bx) as its group sees the frame: A from
    the image, R from `work` for lost samples of earlier-group blocks."""
    H, W = img.shape
    M = B + 2 * d
    f = np.zeros((M, M))
    cls = np.full((M, M), oracle.CLS_OUT, np.uint8)
    g0 = gob[by, bx]
    y0, x0 = by * B - d, bx * B - d
    ys = np.arange(y0, y0 + M)
    xs = np.arange(x0, x0 + M)
    vy = (ys >= 0) & (ys < H)
    vx = (xs >= 0) & (xs < W)
    for mi in np.flatnonzero(vy):
        y = ys[mi]
        for ni in np.flatnonzero(vx):
            x = xs[ni]
            if not mask[y, x]:
                cls[mi, ni] = oracle.CLS_A
                f[mi, ni] = img[y, x]
            elif (y // B, x // B) == (by, bx):
                cls[mi, ni] = oracle.CLS_BI
            elif gob[y // B, x // B] < g0:
                cls[mi, ni] = oracle.CLS_R
                f[mi, ni] = work[y, x]
            else:
                cls[mi, ni] = oracle.CLS_BO
    return f, cls


def trajectory(f, cls, u, rho, delta, gamma, F=64, B=16, d=16, tau_s=TAU_SCALE):
    """Follow the selected indices `u` in FP64.  Returns (worst deficit in
    units of tau, model real part on the centre block [B, B])."""
    w = oracle.weights(cls, rho, delta)
    M = f.shape[0]
    x = np.zeros((F, F))
    x[:M, :M] = w * f
    wp = np.zeros((F, F))
    wp[:M, :M] = w
    R = np.fft.fft2(x)
    Wt = np.fft.fft2(wp)
    W0 = float(w.sum())
    base = float(np.abs(w * f).sum())
    acc = 0.0
    worst = 0.0
    mm, nn = np.mgrid[d:d + B, d:d + B]
    g = np.zeros((B, B), complex)
    for uu in u:
        if uu < 0 or W0 <= 0:
            break
        mag = np.abs(R)
        tau = tau_s * (base + W0 * acc)
        worst = max(worst, (mag.max() - mag.flat[uu]) / tau)
        dc = gamma * R.flat[uu] / W0
        acc += abs(dc)
        um, un = divmod(int(uu), F)
        R = R - dc * np.roll(Wt, (um, un), axis=(0, 1))
        g += dc * np.exp(2j * np.pi * (um * mm + un * nn) / F)
    return worst, g.real


def near_tie_at_divergence(f, cls, u_gpu, u_ref, rho, delta, gamma, F=64, tau_s=TAU_SCALE):
    """At the first index where the trajectories differ, the GPU's pick must
    be a maximiser of |R_w| of the FP64 trajectory within tau.  Returns
    (iteration, deficit / tau)."""
    diff = np.flatnonzero(np.asarray(u_gpu) != np.asarray(u_ref))
    if diff.size == 0:
        return -1, 0.0
    it = int(diff[0])
    r = oracle.extrapolate_area(f, cls, F, it, rho, delta, gamma)
    mag = np.abs(r.R)
    base = float(np.abs(r.w * f).sum())
    W0 = float(r.w.sum())
    tau = tau_s * (base + W0 * float(np.abs(r.dc).sum()))
    return it, float((mag.max() - mag.flat[int(u_gpu[it])]) / tau)
