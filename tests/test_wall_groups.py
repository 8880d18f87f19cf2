"""Host logic of the wall kernel's work units (no GPU): builds tests/native/wall_groups_check.cpp
with the runtime's geometry source (lbcg_geom.cpp) and runs it.  The check covers the
outermost-fluid list of Sec. II.C and the stencil tables of Eq. 28-29 for channels, periodic and
closed boxes and random porous media (see the C++ file)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1707_00198_gb300", "csrc")


def test_wall_groups_resolve_every_neighbour(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "wall_groups_check")
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(ROOT, "tests", "native", "wall_groups_check.cpp"), os.path.join(CSRC, "lbcg_geom.cpp"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout + r.stderr
