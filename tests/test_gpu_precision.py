"""Precision sweep of the projection (DFT-as-GEMM on the tensor cores with
TF32, BF16, FP16 or split-BF16 operands, FP32 accumulation; iterations in
FP32).  The bounds follow from the operand unit roundoff u_P of each type:
the projection's relative error stays within a few u_P, the residual update
stays exact for the spectra it was given, and concealment quality against
the ground truth matches the FP64 oracle's."""
import numpy as np
import pytest

import fse_synth
import oracle
from gpu_util import gpu_conceal, oracle_conceal, psnr

pytestmark = pytest.mark.gpu

# unit roundoff of the operands (8-bit bf16, 11-bit fp16 / tf32 mantissas;
# split bf16 keeps about 16 bits)
U = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11, "bf16x3": 2.0 ** -16,
     "tf32x3": 2.0 ** -21, "fp32": 2.0 ** -22}


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
    yield c
    c.close()


def _prec(fse, name):
    return {"fp32": fse.FSE_PREC_FP32, "tf32": fse.FSE_PREC_TF32, "bf16": fse.FSE_PREC_BF16,
            "fp16": fse.FSE_PREC_FP16, "bf16x3": fse.FSE_PREC_BF16X3,
            "tf32x3": fse.FSE_PREC_TF32X3}[name]


def _areas(n):
    f = np.stack([fse_synth.make_image(48, 48, 900 + i) for i in range(n)]).astype(np.float32)
    cls = np.zeros((n, 48, 48), np.uint8)
    cls[:, 16:32, 16:32] = oracle.CLS_BI
    cls[1::2, 0:16, :] = oracle.CLS_R
    cls[2::4, :, 40:] = oracle.CLS_OUT
    return f, cls


@pytest.mark.parametrize("name", ["fp32", "tf32", "bf16", "fp16", "bf16x3", "tf32x3"])
def test_projection_error_within_operand_precision(fse, ctx, name):
    import torch
    dev = torch.device("cuda:0")
    n = 8
    f, cls = _areas(n)
    p = fse.make_params(iters=0, precision=_prec(fse, name))
    g = torch.empty((n, 16, 16), device=dev)
    r = torch.empty((n, 64, 64, 2), device=dev)
    ctx.fse_extrapolate_areas(torch.from_numpy(f).to(dev), torch.from_numpy(cls).to(dev), p, g,
                              None, None, r)
    torch.cuda.synchronize()
    r = r.cpu().numpy()
    for i in range(n):
        ref = oracle.extrapolate_area(f[i].astype(np.float64), cls[i], 64, 0, 0.7, 0.2, 0.5)
        rel = np.abs(r[i, ..., 0] + 1j * r[i, ..., 1] - ref.R0).max() / np.abs(ref.R0).max()
        assert rel <= 4 * U[name], (name, i, rel)


@pytest.mark.parametrize("name", ["tf32", "bf16", "fp16", "bf16x3", "tf32x3"])
def test_update_consistent_with_its_spectra(fse, ctx, name):
    """Whatever the projection precision, K iterations leave the residual
    equal to DFT{w (f - g)} up to the projection error."""
    import torch
    dev = torch.device("cuda:0")
    n, K = 6, 120
    f, cls = _areas(n)
    p = fse.make_params(iters=K, precision=_prec(fse, name))
    g = torch.empty((n, 16, 16), device=dev)
    u = torch.empty((n, K), dtype=torch.int32, device=dev)
    dc = torch.empty((n, K, 2), device=dev)
    r = torch.empty((n, 64, 64, 2), device=dev)
    ctx.fse_extrapolate_areas(torch.from_numpy(f).to(dev), torch.from_numpy(cls).to(dev), p, g,
                              u, dc, r)
    torch.cuda.synchronize()
    u, dc, r = u.cpu().numpy(), dc.cpu().numpy(), r.cpu().numpy()
    mm, nn = np.mgrid[0:48, 0:48]
    for i in range(n):
        ref = oracle.extrapolate_area(f[i].astype(np.float64), cls[i], 64, 0, 0.7, 0.2, 0.5)
        model = np.zeros((48, 48), complex)
        for uu, d in zip(u[i], dc[i, :, 0] + 1j * dc[i, :, 1]):
            model += d * np.exp(2j * np.pi * ((uu // 64) * mm + (uu % 64) * nn) / 64)
        x = np.zeros((64, 64), complex)
        x[:48, :48] = ref.w * (f[i] - model)
        spatial = np.fft.fft2(x)
        rg = r[i, ..., 0] + 1j * r[i, ..., 1]
        scale = np.abs(ref.R0).max()
        assert np.abs(rg - spatial).max() <= (8 * U[name] + 2e-4) * scale, (name, i)


@pytest.mark.parametrize("name", ["tf32", "bf16", "fp16", "bf16x3", "tf32x3"])
def test_frame_quality_matches_oracle(fse, ctx, name):
    """512x512 mixed losses, K = 200: the reduced-precision projection
    conceals as well as the FP64 oracle against the ground truth (within
    0.3 dB) and stays close to it sample by sample on average."""
    img, mask = fse_synth.workload_mixed_512()[0]
    p = fse.make_params(iters=200, precision=_prec(fse, name))
    (out,), (work,) = gpu_conceal(ctx, [(img, mask)], p)
    o_work, _, _ = oracle_conceal(img, mask, p)
    lost = mask == 1
    gt = img[lost].astype(np.float64)
    q_gpu, q_ora = psnr(work[lost], gt), psnr(o_work[lost], gt)
    print(name, "psnr vs gt", q_gpu, "oracle", q_ora, "psnr vs oracle", psnr(work[lost], o_work[lost]))
    assert abs(q_gpu - q_ora) <= 0.3
    assert psnr(work[lost], o_work[lost]) >= 30.0
    assert np.array_equal(out[~lost], img[~lost])
