"""The iteration-loop microbenchmark (fse_loop_microbench).

Every selecting form of the loop (Sec. 4: u = argmax |R_w|^2, ties to the
smallest index) must pick the same index sequence on the same synthetic
spectra, so their checksums agree; the calibration forms (5, 6) make no
selection and are only checked to run.
"""
import pytest

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


def test_selecting_forms_agree(fse):
    sums = {}
    for v in (0, 1, 2, 3, 4, 7, 8, 9, 10):
        ns, cs = fse.fse_loop_microbench(v, 1, 200, 2, 0)
        assert ns > 0
        sums[v] = cs
    assert len(set(sums.values())) == 1, sums


def test_calibration_forms_run(fse):
    for v in (5, 6):
        ns, _ = fse.fse_loop_microbench(v, 3, 64, 1, 0)
        assert ns > 0


def test_bad_arguments_refused(fse):
    for args in ((11, 1, 200, 2, 0), (0, 0, 200, 2, 0), (0, 1, 0, 2, 0), (0, 1, 200, 0, 0)):
        with pytest.raises(fse.FseError):
            fse.fse_loop_microbench(*args)
