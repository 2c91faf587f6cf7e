"""ctypes binding of ``libfse_gb300.so`` (declared in ``include/fse.h``).

Argument marshalling only: every step of the concealment runs in the native
library.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing or fails to load, import raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfse_gb300.so")

FSE_OK, FSE_EINVAL, FSE_ENOMEM, FSE_EAGAIN, FSE_ETIMEDOUT, FSE_ECUDA, FSE_ENOTFOUND = range(7)
FSE_ETOOBIG = 7
FSE_ORDER_LINESCAN, FSE_ORDER_OPTIMIZED = 0, 1
FSE_PREC_FP32, FSE_PREC_TF32, FSE_PREC_BF16, FSE_PREC_FP16, FSE_PREC_BF16X3, FSE_PREC_TF32X3 = range(6)
FSE_EXEC_GROUPS, FSE_EXEC_PERSISTENT = 0, 1
FSE_MAX_ITERS = 1024

EXPORTED = [
    "fse_plan_order", "fse_plan_claims", "fse_ctx_create", "fse_ctx_destroy", "fse_conceal_batch",
    "fse_conceal_batch_host", "fse_conceal_batch_host_async", "fse_wait_batch",
    "fse_extrapolate_areas", "fse_submit", "fse_poll",
    "fse_drain", "fse_last_batch_info", "fse_last_batch_config", "fse_last_batch_shape", "fse_ctx_set_option", "fse_copy_work", "fse_copy_trace", "fse_last_kernel_ms", "fse_recent_kernel_ms", "fse_last_phase_clocks", "fse_conceal_frame_noalloc", "fse_measure_peaks", "fse_loop_microbench", "fse_weight_table", "fse_strerror",
]
FSE_OPT_SPIN_LIMIT, FSE_OPT_PERSISTENT_CTAS, FSE_OPT_SERVE_SLOTS = 1, 2, 3
FSE_OPT_SERVE_MAX_BATCH, FSE_OPT_TEST_STUCK_DEP, FSE_OPT_KEEP_TRACE = 4, 5, 6
FSE_OPT_GROUP_LAUNCHES, FSE_OPT_AUTOTUNE, FSE_OPT_INPUTS_READY = 7, 8, 9
FSE_OPT_SERVE_LATENCY_MS, FSE_OPT_W_TABLES, FSE_OPT_CLAIM_ORDER = 10, 11, 12
FSE_OPT_PHASE_CLOCKS = 13
FSE_CLAIM_DELAYED, FSE_CLAIM_HEIGHT, FSE_CLAIM_LIST = 0, 1, 2


class fse_params(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("border", ctypes.c_int), ("dft", ctypes.c_int),
                ("iters", ctypes.c_int), ("rho", ctypes.c_float), ("delta", ctypes.c_float),
                ("gamma", ctypes.c_float), ("order", ctypes.c_int), ("precision", ctypes.c_int),
                ("executor", ctypes.c_int)]


class fse_frame(ctypes.Structure):
    _fields_ = [("luma", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("loss_mask", ctypes.c_void_p), ("width", ctypes.c_int),
                ("height", ctypes.c_int), ("stride", ctypes.c_int)]


class fse_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("lost_blocks", ctypes.c_int),
                ("groups", ctypes.c_int), ("batch_requests", ctypes.c_int),
                ("inflight", ctypes.c_int),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class FseError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load the native library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "paper_2207_00233_gb300.build.build() (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, cint = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int
    L.fse_plan_order.argtypes = [cint, cint, vp, cint, vp, vp, vp, ctypes.POINTER(i32)]
    L.fse_plan_claims.argtypes = [cint, vp, vp, vp, cint, cint, cint, vp, vp, ctypes.POINTER(i32)]
    L.fse_measure_peaks.argtypes = [cint, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
    L.fse_loop_microbench.argtypes = [cint, cint, cint, cint, cint,
                                      ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_uint32)]
    L.fse_ctx_create.argtypes = [ctypes.POINTER(vp), cint, ctypes.c_size_t]
    L.fse_ctx_destroy.argtypes = [vp]
    L.fse_ctx_destroy.restype = None
    L.fse_conceal_batch.argtypes = [vp, ctypes.POINTER(fse_frame), cint,
                                    ctypes.POINTER(fse_params), vp]
    L.fse_conceal_batch_host.argtypes = L.fse_conceal_batch.argtypes
    L.fse_conceal_batch_host_async.argtypes = L.fse_conceal_batch.argtypes + [
        ctypes.POINTER(ctypes.c_uint64)]
    L.fse_wait_batch.argtypes = [vp, ctypes.c_uint64]
    L.fse_extrapolate_areas.argtypes = [vp, vp, vp, cint, ctypes.POINTER(fse_params), vp, vp,
                                        vp, vp, vp]
    L.fse_submit.argtypes = [vp, ctypes.POINTER(fse_frame), ctypes.POINTER(fse_params),
                             ctypes.POINTER(ctypes.c_uint64)]
    L.fse_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(cint), ctypes.POINTER(fse_stats)]
    L.fse_drain.argtypes = [vp, cint]
    L.fse_last_batch_config.argtypes = [vp, ctypes.POINTER(cint), ctypes.POINTER(cint)]
    L.fse_last_batch_shape.argtypes = [vp] + [ctypes.POINTER(cint)] * 5
    L.fse_last_phase_clocks.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double), cint,
                                        ctypes.POINTER(cint)]
    L.fse_recent_kernel_ms.argtypes = [vp, cint, vp, ctypes.POINTER(cint)]
    L.fse_last_batch_info.argtypes = [vp, ctypes.POINTER(cint), ctypes.POINTER(cint),
                                      ctypes.POINTER(cint)]
    L.fse_ctx_set_option.argtypes = [vp, cint, ctypes.c_longlong]
    L.fse_weight_table.argtypes = [vp, cint, ctypes.c_float, ctypes.c_float, cint, vp, vp]
    L.fse_copy_work.argtypes = [vp, cint, vp, cint, vp]
    L.fse_copy_trace.argtypes = [vp, cint, vp, vp]
    L.fse_last_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.fse_conceal_frame_noalloc.argtypes = [ctypes.POINTER(fse_frame), ctypes.POINTER(fse_params), vp]
    L.fse_strerror.argtypes = [cint]
    L.fse_strerror.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("fse_ctx_destroy", "fse_strerror"):
            getattr(L, name).restype = cint
    _lib = L
    return L


def strerror(code: int) -> str:
    return lib().fse_strerror(int(code)).decode()


def _check(rc: int, where: str) -> None:
    if rc != FSE_OK:
        raise FseError(rc, where)


def _host_frames(frames):
    """fse_frame array of host (luma, mask, out) uint8 arrays or CPU tensors."""
    arr = (fse_frame * len(frames))()
    for i, (luma, mask, out) in enumerate(frames):
        ptrs = []
        for a in (luma, mask, out):
            if isinstance(a, np.ndarray):
                if a.dtype != np.uint8 or not a.flags["C_CONTIGUOUS"] or a.ndim != 2:
                    raise ValueError("host frames must be C-contiguous 2-D uint8 arrays")
                ptrs.append(a.ctypes.data)
            else:
                if not a.is_contiguous() or a.dim() != 2:
                    raise ValueError("host tensors must be contiguous 2-D")
                ptrs.append(a.data_ptr())
        h, w = luma.shape
        arr[i] = fse_frame(ptrs[0], ptrs[2], ptrs[1], w, h, w)
    return arr


def make_params(iters: int = 200, rho: float = 0.7, delta: float = 0.2, gamma: float = 0.5,
                order: int = FSE_ORDER_OPTIMIZED, precision: int = FSE_PREC_FP32,
                executor: int = FSE_EXEC_PERSISTENT, block: int = 16, border: int = 16,
                dft: int = 64) -> fse_params:
    return fse_params(block, border, dft, iters, rho, delta, gamma, order, precision, executor)


def fse_plan_order(block_lost: np.ndarray, order: int):
    """Processing order of one frame.  Returns (group_of_block [BH, BW],
    group_ptr [G+1], block_ids [lost blocks]) as int32 arrays."""
    lost = np.ascontiguousarray(block_lost, dtype=np.uint8)
    if lost.ndim != 2:
        raise ValueError("block_lost must be 2-D [BH, BW]")
    bh, bw = lost.shape
    nb = bh * bw
    gob = np.empty(nb, np.int32)
    gptr = np.zeros(nb + 1, np.int32)
    ids = np.zeros(max(nb, 1), np.int32)
    ng = ctypes.c_int32(0)
    _check(lib().fse_plan_order(bw, bh, lost.ctypes.data, int(order), gob.ctypes.data,
                                gptr.ctypes.data, ids.ctypes.data, ctypes.byref(ng)),
           "fse_plan_order")
    n = ng.value
    return gob.reshape(bh, bw), gptr[:n + 1].copy(), ids[:int(gptr[n])].copy()


def fse_measure_peaks(device: int = 0):
    """Measured shared-memory load bandwidth (GB/s) and packed FP32 FMA
    throughput (TFLOP/s) of the device."""
    smem, fp32 = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().fse_measure_peaks(int(device), ctypes.byref(smem), ctypes.byref(fp32)),
           "fse_measure_peaks")
    return smem.value, fp32.value


def fse_loop_microbench(variant: int, ctas_per_sm: int, iters: int = 200,
                        blocks_per_cta: int = 8, device: int = 0):
    """Iteration loop alone: (ns per block-iteration per SM, checksum of the
    selected indices)."""
    ns, cs = ctypes.c_double(0), ctypes.c_uint32(0)
    _check(lib().fse_loop_microbench(int(device), int(variant), int(ctas_per_sm), int(iters),
                                     int(blocks_per_cta), ctypes.byref(ns), ctypes.byref(cs)),
           "fse_loop_microbench")
    return ns.value, cs.value


def fse_plan_claims(group_maps, block: int = 16, workers: int = 0, mode: int = 0):
    """Claim order of the lost blocks of several frames (group maps as from
    fse_plan_order).  Returns (items [L, 2] int32 (frame, block), level_start
    [levels + 1] or None in mode 1)."""
    maps = [np.ascontiguousarray(g, dtype=np.int32) for g in group_maps]
    bw = np.array([g.shape[1] for g in maps], np.int32)
    bh = np.array([g.shape[0] for g in maps], np.int32)
    flat = np.concatenate([g.ravel() for g in maps]) if maps else np.zeros(0, np.int32)
    lost = int((flat >= 0).sum())
    items = np.zeros((max(lost, 1), 2), np.int32)
    level_start = np.zeros(lost + 2, np.int32)
    nl = ctypes.c_int32(0)
    _check(lib().fse_plan_claims(len(maps), bw.ctypes.data, bh.ctypes.data, flat.ctypes.data,
                                 int(block), int(workers), int(mode), items.ctypes.data,
                                 level_start.ctypes.data, ctypes.byref(nl)),
           "fse_plan_claims")
    return items[:lost].copy(), (level_start[:nl.value + 1].copy() if mode == 0 else None)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """Owns one ``fse_ctx``."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        h = ctypes.c_void_p()
        _check(lib().fse_ctx_create(ctypes.byref(h), int(device), int(mem_budget)),
               "fse_ctx_create")
        self.handle = h

    def close(self) -> None:
        if self.handle:
            lib().fse_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- device frames (torch CUDA uint8 tensors [H, W]) --------------------
    @staticmethod
    def _frames_from_tensors(frames):
        arr = (fse_frame * len(frames))()
        for i, (luma, mask, out) in enumerate(frames):
            for t in (luma, mask, out):
                if t.dtype.itemsize != 1 or t.dim() != 2 or t.stride(1) != 1:
                    raise ValueError("frames must be 2-D uint8 tensors with unit column stride")
            if luma.shape != mask.shape or luma.shape != out.shape:
                raise ValueError("luma, mask and out must have the same shape")
            if luma.stride(0) != mask.stride(0) or luma.stride(0) != out.stride(0):
                raise ValueError("luma, mask and out must share the row stride")
            h, w = luma.shape
            arr[i] = fse_frame(luma.data_ptr(), out.data_ptr(), mask.data_ptr(), w, h,
                               luma.stride(0))
        return arr

    def fse_conceal_batch(self, frames, params: fse_params, stream=None) -> None:
        """frames: list of (luma, mask, out) CUDA uint8 tensors."""
        arr = self._frames_from_tensors(frames)
        _check(lib().fse_conceal_batch(self.handle, arr, len(frames), ctypes.byref(params),
                                       _stream_handle(stream)), "fse_conceal_batch")

    def fse_conceal_batch_host(self, frames, params: fse_params, stream=None) -> None:
        """frames: list of (luma, mask, out) C-contiguous uint8 numpy arrays
        (or pinned CPU tensors); out is written before the call returns."""
        _check(lib().fse_conceal_batch_host(self.handle, _host_frames(frames), len(frames),
                                            ctypes.byref(params), _stream_handle(stream)),
               "fse_conceal_batch_host")

    def fse_conceal_batch_host_async(self, frames, params: fse_params, stream=None) -> int:
        """As fse_conceal_batch_host, but returns a ticket once the batch is
        enqueued; the buffers must stay alive until fse_wait_batch(ticket)."""
        t = ctypes.c_uint64(0)
        _check(lib().fse_conceal_batch_host_async(self.handle, _host_frames(frames), len(frames),
                                                  ctypes.byref(params), _stream_handle(stream),
                                                  ctypes.byref(t)),
               "fse_conceal_batch_host_async")
        return t.value

    def fse_wait_batch(self, ticket: int) -> None:
        _check(lib().fse_wait_batch(self.handle, ctypes.c_uint64(ticket)), "fse_wait_batch")

    def fse_extrapolate_areas(self, area_f, area_cls, params: fse_params, g_out, u_out=None,
                              dc_out=None, r_out=None, stream=None) -> None:
        """CUDA tensors: area_f float32 [n,48,48], area_cls uint8 [n,48,48],
        g_out float32 [n,16,16]; optional u_out int32 [n,K], dc_out float32
        [n,K,2], r_out float32 [n,64,64,2]."""
        n = area_f.shape[0]
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(lib().fse_extrapolate_areas(self.handle, area_f.data_ptr(), area_cls.data_ptr(),
                                           n, ctypes.byref(params), g_out.data_ptr(),
                                           ptr(u_out), ptr(dc_out), ptr(r_out),
                                           _stream_handle(stream)), "fse_extrapolate_areas")

    def fse_submit(self, luma: np.ndarray, mask: np.ndarray, out: np.ndarray,
                   params: fse_params) -> int:
        """Queue one host frame; the arrays must stay alive until done."""
        for a in (luma, mask, out):
            if a.dtype != np.uint8 or not a.flags["C_CONTIGUOUS"] or a.ndim != 2:
                raise ValueError("serving frames must be C-contiguous 2-D uint8 arrays")
        h, w = luma.shape
        fr = fse_frame(luma.ctypes.data, out.ctypes.data, mask.ctypes.data, w, h, w)
        t = ctypes.c_uint64(0)
        rc = lib().fse_submit(self.handle, ctypes.byref(fr), ctypes.byref(params), ctypes.byref(t))
        if rc == FSE_EAGAIN:
            return -1
        _check(rc, "fse_submit")
        return int(t.value)

    def fse_poll(self, ticket: int):
        """Returns None while running, else the fse_stats of the request."""
        done = ctypes.c_int(0)
        st = fse_stats()
        _check(lib().fse_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(done),
                              ctypes.byref(st)), "fse_poll")
        return st if done.value else None

    def fse_drain(self, timeout_ms: int = -1) -> None:
        _check(lib().fse_drain(self.handle, int(timeout_ms)), "fse_drain")

    def fse_copy_trace(self, frame: int, dst, stream=None) -> None:
        """dst: CUDA int16 tensor with bh*bw*iters elements."""
        _check(lib().fse_copy_trace(self.handle, int(frame), dst.data_ptr(),
                                    _stream_handle(stream)), "fse_copy_trace")

    def fse_last_kernel_ms(self) -> float:
        ms = ctypes.c_float(0.0)
        _check(lib().fse_last_kernel_ms(self.handle, ctypes.byref(ms)), "fse_last_kernel_ms")
        return float(ms.value)

    def fse_copy_work(self, frame: int, dst, stream=None) -> None:
        """dst: CUDA float32 tensor [H, >=W] with unit column stride."""
        _check(lib().fse_copy_work(self.handle, int(frame), dst.data_ptr(), dst.stride(0),
                                   _stream_handle(stream)), "fse_copy_work")

    def fse_ctx_set_option(self, option: int, value: int) -> None:
        _check(lib().fse_ctx_set_option(self.handle, int(option), int(value)),
               "fse_ctx_set_option")

    def fse_weight_table(self, key: int, rho: float, delta: float, builder: int, dst,
                         stream=None) -> None:
        """W table of class pattern `key` into the device tensor dst (float32,
        71 x 64 x 4 elements); builder 1 = FP32 split DFTs, 2 = tensor cores."""
        _check(lib().fse_weight_table(self.handle, int(key), float(rho), float(delta),
                                      int(builder), ctypes.c_void_p(dst.data_ptr()),
                                      ctypes.c_void_p(_stream_handle(stream))),
               "fse_weight_table")

    def fse_recent_kernel_ms(self, n: int):
        """Kernel times (ms) of the last n batches, most recent first."""
        buf = (ctypes.c_float * max(n, 1))()
        cnt = ctypes.c_int(0)
        _check(lib().fse_recent_kernel_ms(self.handle, int(n), buf, ctypes.byref(cnt)),
               "fse_recent_kernel_ms")
        return [buf[j] for j in range(cnt.value)]

    def fse_last_batch_config(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().fse_last_batch_config(self.handle, ctypes.byref(a), ctypes.byref(b)),
               "fse_last_batch_config")
        return {"executor": a.value, "ctas_per_sm": b.value}

    PHASES = ("wait", "staging", "gather", "projection", "iterations", "synthesis", "store")

    def fse_last_phase_clocks(self, stream=None):
        """Mean SM clocks per block of each phase of the last persistent batch
        (FSE_OPT_PHASE_CLOCKS) and the number of blocks averaged."""
        buf = (ctypes.c_double * 7)()
        cnt = ctypes.c_int(0)
        _check(lib().fse_last_phase_clocks(self.handle, ctypes.c_void_p(_stream_handle(stream)),
                                           buf, 7, ctypes.byref(cnt)), "fse_last_phase_clocks")
        return dict(zip(self.PHASES, list(buf))), cnt.value

    def fse_last_batch_shape(self):
        v = [ctypes.c_int() for _ in range(5)]
        _check(lib().fse_last_batch_shape(self.handle, *[ctypes.byref(x) for x in v]),
               "fse_last_batch_shape")
        return dict(zip(("executor", "ctas_per_sm", "claim_order", "threads_per_cta",
                         "blocks_per_cta"), (x.value for x in v)))

    def fse_last_batch_info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().fse_last_batch_info(self.handle, ctypes.byref(a), ctypes.byref(b),
                                         ctypes.byref(c)), "fse_last_batch_info")
        return {"lost_blocks": a.value, "groups": b.value, "launches": c.value}
