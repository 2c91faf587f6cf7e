"""Host-side tests of the native library (no GPU needed).

The library must build with nvcc here (cross-compiled for sm_103a), load,
and export every entry point that include/fse.h declares.  The processing
order (Algorithm 1, Sec. 3) is host code: it is checked bit for bit against
the oracle's independent implementation on many random loss maps.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fse():
    from paper_2207_00233_gb300 import build
    build.build()
    import paper_2207_00233_gb300 as pkg
    pkg.lib()
    return pkg


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "fse.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[a-z][\w \*]*?\b(fse_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(fse):
    names = _declared_symbols()
    assert len(names) >= 12
    L = fse.lib()
    for name in names:
        assert hasattr(L, name), name
        assert isinstance(getattr(L, name), ctypes._CFuncPtr)
    assert sorted(fse.EXPORTED) == names


def test_strerror(fse):
    assert fse.strerror(0) == "ok"
    assert "invalid" in fse.strerror(1)
    assert fse.strerror(999) == "unknown status"


@pytest.mark.parametrize("order", [0, 1])
def test_plan_matches_oracle_on_golden_shapes(fse, order):
    for shape, cells in [((5, 5), (slice(1, 4), slice(1, 4))), ((8, 8), (3, slice(None))),
                         ((3, 3), (slice(None), slice(None)))]:
        lost = np.zeros(shape, np.uint8)
        lost[cells] = 1
        a = fse.fse_plan_order(lost, order)
        b = oracle.plan(lost, order)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_plan_fuzz_bit_exact_against_oracle(fse):
    rng = np.random.default_rng(1234)
    for trial in range(10000):
        bh = int(rng.integers(1, 24))
        bw = int(rng.integers(1, 24))
        kind = trial % 4
        if kind == 0:
            lost = rng.random((bh, bw)) < rng.uniform(0.0, 1.0)
        elif kind == 1:  # bursts along rows
            lost = np.zeros((bh, bw), bool)
            for _ in range(int(rng.integers(0, 6))):
                r = int(rng.integers(0, bh))
                c = int(rng.integers(0, bw))
                lost[r, c:c + int(rng.integers(1, 9))] = True
        elif kind == 2:  # full slices
            lost = rng.random((bh, bw)) < 0.1
            lost[int(rng.integers(0, bh)), :] = True
        else:
            lost = rng.random((bh, bw)) < 0.9
        lost = lost.astype(np.uint8)
        order = int(trial % 2)
        a = fse.fse_plan_order(lost, order)
        b = oracle.plan(lost, order)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), (trial, bh, bw)


@pytest.mark.parametrize("bh,bw", [(68, 120), (135, 240), (18, 22)])
def test_plan_bit_exact_frame_sizes(fse, bh, bw):
    rng = np.random.default_rng(bh * 1000 + bw)
    for rate in (0.05, 0.25, 0.5, 0.95):
        lost = (rng.random((bh, bw)) < rate).astype(np.uint8)
        for order in (0, 1):
            a = fse.fse_plan_order(lost, order)
            b = oracle.plan(lost, order)
            for x, y in zip(a, b):
                assert np.array_equal(x, y)


def test_plan_rejects_bad_arguments(fse):
    with pytest.raises(fse.FseError) as e:
        fse.fse_plan_order(np.zeros((2, 2), np.uint8), 7)
    assert e.value.code == 1
    L = fse.lib()
    n = ctypes.c_int32()
    assert L.fse_plan_order(0, 3, None, 1, None, None, None, ctypes.byref(n)) == 1


def test_no_gpu_context_fails_cleanly(fse):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fse.FseError):
        fse.Context(0)


def test_package_has_no_cpu_fallback():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2207_00233_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower().replace("oracle_", ""), f
