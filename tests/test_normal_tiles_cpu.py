"""Host logic of the row-tile normal product (no GPU): the plan built by
csrc/normal_tiles.cpp, compiled with the host compiler together with
tests/normal_tiles_check.cpp, reproduces w = A^T (A p) from its definition on several
matrices (a banded one, empty rows and columns, a full-width row, a 1 x 1 matrix, rows in
no order) and refuses a row wider than a block's shared memory."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_row_tile_plan(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "normal_tiles_check")
    src = [os.path.join(ROOT, "tests", "normal_tiles_check.cpp"),
           os.path.join(ROOT, "paper_2107_09006_gb300", "csrc", "normal_tiles.cpp")]
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-o", exe] + src, check=True, capture_output=True,
                   text=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(p.stdout)
    assert p.returncode == 0 and "ALL OK" in p.stdout, p.stdout + p.stderr
