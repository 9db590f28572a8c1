"""Index maps of the label tiles (Sec. 5.2 path compression over tiles):
the halo shell's and the face cells' index maps are bijections onto the
cells they name, exit-table slots are distinct per face vertex, and every
shell cell inside the grid has a slot (tests/label_geometry_check.cu,
compiled for the host with nvcc and run here; no GPU needed)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_label_geometry_maps():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "geomcheck")
        r = subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-I", os.path.join(ROOT, "include"),
                            "-I", os.path.join(ROOT, "paper_2406_09423_gb300", "csrc"),
                            "-o", exe, os.path.join(ROOT, "tests", "label_geometry_check.cu")],
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "0 problems" in r.stdout
