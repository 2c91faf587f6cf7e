"""The C-ABI from a plain C99 program: include/fse.h compiles as C with
warnings as errors, the program links against the library, and the
processing order it prints for each hand-derived golden grid (Sec. 3,
Algorithm 1) matches the golden file."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_2207_00233_gb300 import build
    build.build()
    from paper_2207_00233_gb300 import _native
    libdir = os.path.dirname(_native.LIB_PATH)
    out = str(tmp_path_factory.mktemp("c_abi") / "plan_from_c")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "plan_from_c.c"),
           "-o", out, "-L", libdir, "-l:" + os.path.basename(_native.LIB_PATH),
           "-Wl,-rpath," + libdir]
    subprocess.run(cmd, check=True)
    return out


def _grid(text):
    rows = [ln.split() for ln in text.splitlines() if ln.strip() and not ln.startswith("#")]
    assert rows[0][0] == "grid"
    return [list(map(int, r)) for r in rows[1:]]


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(GOLDEN) if f.startswith("schedule_")))
def test_plan_from_c_matches_golden(exe, name):
    text = open(os.path.join(GOLDEN, name)).read()
    grid_text = "\n".join(ln for ln in text.splitlines() if not ln.startswith("#"))
    res = subprocess.run([exe, "1"], input=grid_text, capture_output=True, text=True, timeout=60)
    assert res.returncode == 0, res.stderr
    assert _grid(res.stdout) == _grid(text)


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(GOLDEN) if f.startswith("schedule_")))
def test_linescan_from_c_is_raster_rank(exe, name):
    """Line scan: one group per lost block, in raster order."""
    text = open(os.path.join(GOLDEN, name)).read()
    grid_text = "\n".join(ln for ln in text.splitlines() if not ln.startswith("#"))
    res = subprocess.run([exe, "0"], input=grid_text, capture_output=True, text=True, timeout=60)
    assert res.returncode == 0, res.stderr
    rank, want = 0, []
    for row in _grid(text):
        out = []
        for g in row:
            out.append(rank if g >= 0 else -1)
            rank += g >= 0
        want.append(out)
    assert _grid(res.stdout) == want
