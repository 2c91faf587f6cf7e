"""Weight-spectrum tables (FSE_OPT_W_TABLES, fse_weight_table).

A block lost as a whole whose eight neighbours are each not lost, lost as a
whole, or outside the image has its sub-area classes (Sec. 2, Fig. 1) fixed
by a 16-bit key, and W = DFT64 of its Eq. (2) weights with them.  The tables
of both builders (the blocks' FP32 split DFTs, and DFT-as-GEMM on the tcgen05
tensor cores with split-TF32 operands) are checked against numpy's FFT of
the oracle's weights for hand-built class grids, for exact conjugate
symmetry and for the W4 layout; concealment with tensor-core tables meets
the parity criterion against the oracle.
"""
import numpy as np
import pytest

import fse_synth
import oracle
from gpu_util import gpu_conceal, run_and_compare

pytestmark = pytest.mark.gpu

A, R, BI, BO, OUT = oracle.CLS_A, oracle.CLS_R, oracle.CLS_BI, oracle.CLS_BO, oracle.CLS_OUT
# neighbour order of the key: (dy, dx) in raster order without the centre
NEIGHBOURS = [(0, 0), (0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1), (2, 2)]
STATE_CLASS = {0: A, 1: R, 2: BO, 3: OUT}


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


def classes_of_key(key):
    cls = np.empty((48, 48), np.uint8)
    cls[16:32, 16:32] = BI
    for j, (cy, cx) in enumerate(NEIGHBOURS):
        cls[16 * cy:16 * cy + 16, 16 * cx:16 * cx + 16] = STATE_CLASS[(key >> (2 * j)) & 3]
    return cls


def reference_w(key, rho, delta):
    w = oracle.weights(classes_of_key(key), rho, delta)
    x = np.zeros((64, 64))
    x[:48, :48] = w
    return np.fft.fft2(x), float(w.sum())


def gpu_table(fse, ctx, key, rho, delta, builder):
    import torch
    t = torch.empty((71, 64, 4), dtype=torch.float32, device="cuda:0")
    ctx.fse_weight_table(key, rho, delta, builder, t)
    torch.cuda.synchronize()
    return t.cpu().numpy()


def unpack_w4(t):
    """W4 rows 0..63 -> complex W[64, 64] (from the direct columns)."""
    return t[:64, :, 0] + 1j * t[:64, :, 2]


KEYS = [0, 0xFFFF, 0x5555, 0xAAAA,
        # a corner of the image: the upper row and the left column outside
        (3 << 0) | (3 << 2) | (3 << 4) | (3 << 6) | (3 << 10),
        # earlier-group neighbours above, later-group below, support beside
        (1 << 0) | (1 << 2) | (1 << 4) | (2 << 10) | (2 << 12) | (2 << 14)]
KEYS += [int(k) for k in np.random.default_rng(5).integers(0, 1 << 16, 6)]


@pytest.mark.parametrize("builder", [1, 2])
@pytest.mark.parametrize("rho,delta", [(0.7, 0.2), (0.8, 0.2), (0.5, 0.9)])
def test_table_matches_library_dft(fse, ctx, builder, rho, delta):
    worst = [0.0]
    for key in KEYS:
        t = gpu_table(fse, ctx, key, rho, delta, builder)
        ref, w0 = reference_w(key, rho, delta)
        got = unpack_w4(t)
        # FP32-grade: every entry is a sum of weights times unit phases, so
        # its rounding scales with W[0] = sum w; two DFT stages of 48-term
        # sums (and, on the tensor cores, split-TF32 products good to about
        # 2^-21 each) stay within 2^-19 W[0]
        scale = max(w0, 1e-30)
        err = float(np.abs(got - ref).max()) / scale
        worst[0] = max(worst[0], err)
        assert err <= 2.0 ** -19, (builder, hex(key), err)
        # W4 layout: the partner column and the repeated rows
        assert np.array_equal(t[:64, :, 1], t[:64, np.arange(64) ^ 32, 0])
        assert np.array_equal(t[:64, :, 3], t[:64, np.arange(64) ^ 32, 2])
        assert np.array_equal(t[64:71], t[0:7])
    print(f"builder {builder}: worst |W - FFT| / W[0] = {worst[0]:.3e} "
          f"({worst[0] / 2.0 ** -24:.1f} x 2^-24)")


@pytest.mark.parametrize("builder", [1, 2])
def test_table_exactly_conjugate_symmetric(fse, ctx, builder):
    """Real weights give W[-k] = conj W[k]; the tables keep it bit for bit
    (the iterations rely on it for the exact ties of real spectra)."""
    neg = (-np.arange(64)) % 64
    for key in KEYS:
        w = unpack_w4(gpu_table(fse, ctx, key, 0.7, 0.2, builder))
        mirror = w[np.ix_(neg, neg)]
        assert np.array_equal(mirror.real, w.real) and np.array_equal(mirror.imag, -w.imag), \
            (builder, hex(key))


def test_tensor_tables_conceal_within_parity(fse, ctx):
    """The default tables (tensor cores) on the 512x512 mixed-loss frame and
    a 1920x1080 frame of the batch: the parity criterion of the FP32 path."""
    ctx.fse_ctx_set_option(fse.FSE_OPT_W_TABLES, 2)
    frames = fse_synth.workload_mixed_512() + fse_synth.workload_batch_1080p(1)
    p = fse.make_params(iters=200, order=fse.FSE_ORDER_OPTIMIZED,
                        executor=fse.FSE_EXEC_PERSISTENT)
    *_, stats = run_and_compare(ctx, frames, p, "tensor-core tables")
    print(stats)


def test_tensor_tables_close_to_fp32_tables(fse):
    """Outputs with tensor-core tables against FP32 tables: the FP32 working
    values of every block agree within the pixel tolerance, or the block's
    selection trace differs (a near-tie the two roundings resolve apart)."""
    frames = fse_synth.workload_batch_1080p(2)
    p = fse.make_params(iters=200, order=fse.FSE_ORDER_OPTIMIZED,
                        executor=fse.FSE_EXEC_PERSISTENT)
    res = []
    for builder in (1, 2):
        with fse.Context(0) as c:
            c.fse_ctx_set_option(fse.FSE_OPT_W_TABLES, builder)
            res.append(gpu_conceal(c, frames, p))
    for (o1, w1), (o2, w2) in [((res[0][0][i], res[0][1][i]), (res[1][0][i], res[1][1][i]))
                               for i in range(len(frames))]:
        lost = ~np.isnan(w1)
        d = np.abs(w1[lost] - w2[lost])
        # most samples agree to FP32 rounding; the rest come from near-ties
        assert np.mean(d <= 0.5) >= 0.8, np.mean(d <= 0.5)
        assert np.array_equal(o1[~lost], o2[~lost])
