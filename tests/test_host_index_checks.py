"""Host checks of the index arithmetic the device kernels rely on: the
gather tiles of K and K^T, the pre-wrapped ray taps, the segment table and the
per-direction planes of coupling selection and the edge form,
computed with the library's own graph and view builders for several grid
shapes (tests/host/index_checks.cpp, built here with the host compiler)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_16037_gb300", "csrc")


def test_device_indices_land_in_bounds_and_on_the_right_nodes(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "index_checks")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host", "index_checks.cpp"),
                    os.path.join(CSRC, "graph.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    print(out.stdout)
    assert out.returncode == 0, out.stdout + out.stderr
