"""Host checks of the gridding plan (no GPU): the C++ planning code of the
library, compiled here with the host compiler, is run on seeded footprint
layouts and checked against brute force (sort, tile lists, work units, the
stored gather walk) and against the scatter form of G^T (§5: G sparse and
fixed by the frequencies)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1307_4370_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("plan") / "gather_plan_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "gather_plan_check.cpp"),
                    os.path.join(CSRC, "gather_plan.cpp"), "-o", exe], check=True)
    return exe


# (grid side L, footprint J, tile T, visibilities M, layout, seed); layouts:
# 0 uniform, 1 half on three dense cells (multi-chunk tiles), 2 at the wrap edges
CASES = [
    (128, 4, 16, 2048, 0, 1),
    (128, 6, 16, 6000, 1, 2),
    (128, 6, 32, 6000, 2, 3),
    (64, 8, 16, 3000, 1, 4),
    (96, 6, 16, 4000, 0, 5),   # 3 * 2^k grid side
    (128, 2, 64, 5000, 1, 6),
    (64, 6, 16, 0, 0, 7),      # no visibilities
    (64, 6, 16, 1, 2, 8),
    (256, 6, 16, 40000, 1, 9),
]


@pytest.mark.parametrize("L,J,T,M,layout,seed", CASES)
def test_gather_plan(checker, L, J, T, M, layout, seed):
    r = subprocess.run([checker, str(L), str(J), str(T), str(M), str(layout), str(seed)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
