"""Python access to the FP64 CPU oracle (``fse_oracle.c``) through ctypes.

TEST INFRASTRUCTURE ONLY.  Imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark.  The product package never imports
this module, and this module never imports the product package.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

CLS_A, CLS_R, CLS_BI, CLS_BO, CLS_OUT = 0, 1, 2, 3, 4
ORDER_LINESCAN, ORDER_OPTIMIZED = 0, 1

_lib = None

_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


class _OptPtr:
    """ctypes argument type accepting a C-contiguous ndarray or None."""

    @classmethod
    def from_param(cls, obj):
        if obj is None:
            return ctypes.c_void_p(None)
        if not obj.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(obj.ctypes.data)


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_plan.argtypes = [ctypes.c_int, ctypes.c_int, _u8p, ctypes.c_int,
                                  _i32p, _i32p, _i32p, ctypes.POINTER(ctypes.c_int32)]
        L.oracle_plan.restype = ctypes.c_int
        L.oracle_weights.argtypes = [ctypes.c_int, ctypes.c_int, _u8p, ctypes.c_double,
                                     ctypes.c_double, _f64p]
        L.oracle_weights.restype = None
        L.oracle_extrapolate_area.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p, _u8p,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
            _OptPtr, _OptPtr, _OptPtr, _OptPtr, _OptPtr, _OptPtr, _OptPtr, _OptPtr, _OptPtr,
            _OptPtr]
        L.oracle_extrapolate_area.restype = ctypes.c_int
        L.oracle_conceal_frame.argtypes = [
            ctypes.c_int, ctypes.c_int, _u8p, _u8p, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, _f64p, _u8p, _OptPtr, _OptPtr]
        L.oracle_conceal_frame.restype = ctypes.c_int
        L.oracle_conceal_frame_ex.argtypes = L.oracle_conceal_frame.argtypes + [_OptPtr, _OptPtr]
        L.oracle_conceal_frame_ex.restype = ctypes.c_int
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def plan(lost_blocks: np.ndarray, order: int):
    """Processing order (line scan or Algorithm 1) for a [BH, BW] loss map.

    Returns (group_of_block [BH, BW] int32, group_ptr int32, block_ids int32).
    """
    lost = np.ascontiguousarray(lost_blocks, dtype=np.uint8)
    bh, bw = lost.shape
    nb = bh * bw
    gob = np.empty(nb, np.int32)
    gptr = np.zeros(nb + 1, np.int32)
    ids = np.zeros(max(nb, 1), np.int32)
    ng = ctypes.c_int32(0)
    rc = lib().oracle_plan(bw, bh, lost.ravel(), int(order), gob, gptr, ids, ctypes.byref(ng))
    if rc:
        raise ValueError(f"oracle_plan failed ({rc})")
    n = int(ng.value)
    return gob.reshape(bh, bw), gptr[:n + 1].copy(), ids[:int(gptr[n])].copy()


def weights(cls: np.ndarray, rho: float, delta: float) -> np.ndarray:
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    M, N = cls.shape
    w = np.empty((M, N), np.float64)
    lib().oracle_weights(M, N, cls.ravel(), float(rho), float(delta), w.ravel())
    return w


@dataclass
class AreaResult:
    g: np.ndarray       # [M, N] real part of the model over the whole area
    w: np.ndarray       # [M, N] weights
    R0: np.ndarray      # [F, F] complex initial weighted residual spectrum
    W: np.ndarray       # [F, F] complex spectrum of the weights
    u: np.ndarray       # [K] selected linear index F*k_m + k_n
    dc: np.ndarray      # [K] complex coefficient increments
    R: np.ndarray       # [F, F] complex final weighted residual spectrum
    coef: np.ndarray    # [F, F] complex expansion coefficients
    margin: np.ndarray  # [K] selection margins (see fse_oracle.h)


def extrapolate_area(f: np.ndarray, cls: np.ndarray, F: int, K: int, rho: float,
                     delta: float, gamma: float, tie_largest: bool = False,
                     want_g: np.ndarray | None = None) -> AreaResult:
    """FSE of one area with every intermediate quantity returned."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    M, N = f.shape
    g = np.zeros((M, N), np.float64)
    w = np.empty((M, N), np.float64)
    R0 = np.empty((F, F, 2), np.float64)
    W = np.empty((F, F, 2), np.float64)
    u = np.empty(max(K, 1), np.int32)
    dc = np.empty((max(K, 1), 2), np.float64)
    R = np.empty((F, F, 2), np.float64)
    coef = np.empty((F, F, 2), np.float64)
    margin = np.empty(max(K, 1), np.float64)
    wg = None if want_g is None else np.ascontiguousarray(want_g, dtype=np.uint8)
    rc = lib().oracle_extrapolate_area(M, N, F, f, cls, rho, delta, gamma, K,
                                       1 if tie_largest else 0, wg, g, w, R0, W, u, dc, R, coef,
                                       margin)
    if rc:
        raise ValueError(f"oracle_extrapolate_area failed ({rc})")

    def cplx(a):
        return a[..., 0] + 1j * a[..., 1]

    return AreaResult(g=g, w=w, R0=cplx(R0), W=cplx(W), u=u[:K].copy(),
                      dc=cplx(dc[:K]), R=cplx(R), coef=cplx(coef), margin=margin[:K].copy())


def conceal_frame(img: np.ndarray, mask: np.ndarray, *, block: int = 16, border: int = 16,
                  dft: int = 64, iters: int = 200, rho: float = 0.7, delta: float = 0.2,
                  gamma: float = 0.5, order: int = ORDER_OPTIMIZED, threads: int = 1,
                  trace: bool = False, classes: bool = False, margins: bool = False):
    """Conceal one frame.  Returns (work FP64 [H,W], out uint8 [H,W],
    group_of_block int32 [BH,BW]), plus the selection trace
    [BH*BW, iters] int32 (-2 for blocks without loss) when ``trace``, the
    sub-area classes of every concealed block's area [BH*BW, M, M] uint8
    (255 for blocks without loss) when ``classes``, and the selection
    margins [BH*BW, iters] float64 (inf for blocks without loss) when
    ``margins``."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    H, Wd = img.shape
    if mask.shape != img.shape:
        raise ValueError("mask shape differs from image shape")
    bh, bw = (H + block - 1) // block, (Wd + block - 1) // block
    work = np.empty((H, Wd), np.float64)
    out = np.empty((H, Wd), np.uint8)
    gob = np.empty((bh, bw), np.int32)
    ut = np.full((bh * bw, max(iters, 1)), -2, np.int32) if trace else None
    M = block + 2 * border
    ct = np.full((bh * bw, M, M), 255, np.uint8) if classes else None
    mt = np.full((bh * bw, max(iters, 1)), np.inf) if margins else None
    rc = lib().oracle_conceal_frame_ex(H, Wd, img.ravel(), mask.ravel(), block, border, dft,
                                       iters, rho, delta, gamma, int(order), int(threads),
                                       work.ravel(), out.ravel(), gob, ut, ct, mt)
    if rc:
        raise ValueError(f"oracle_conceal_frame failed ({rc})")
    res = [work, out, gob]
    if trace:
        res.append(ut[:, :iters])
    if classes:
        res.append(ct)
    if margins:
        res.append(mt[:, :iters])
    return tuple(res)
