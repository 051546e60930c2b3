"""The bounds-checked build (-DFEMPIC_CHECKS=1) compiles for sm_103a on the
CPU: tet ids from a caller's device buffer (before they are copied) and in
the particle kernels, and the per-tet DOF and neighbour tables at create, are
range-checked; an out-of-range index sets the device status
word (FEMPIC_ERR_BOUNDS) instead of being read.  Both the checked and the
default translation unit export the table check's launch stub."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.mark.skipif(not (os.path.exists(NVCC) or shutil.which("nvcc")), reason="nvcc not found")
def test_checked_build_compiles(tmp_path):
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    obj = tmp_path / "fempic_checked.o"
    subprocess.run([nvcc, "-O3", "-std=c++17", "-gencode=arch=compute_103a,code=sm_103a", "-Xcompiler",
                    "-fPIC,-ffp-contract=off", "-I", os.path.join(ROOT, "include"), "-DFEMPIC_CHECKS=1", "-c",
                    os.path.join(ROOT, "paper_2111_12411_gb300", "csrc", "fempic.cu"), "-o", str(obj)],
                   check=True, capture_output=True)
    syms = subprocess.run(["nm", "-C", str(obj)], check=True, capture_output=True, text=True).stdout
    assert "k_check_tables" in syms and "k_check_ids" in syms and "femPIC_step" in syms


def test_bounds_error_code_is_exported():
    from paper_2111_12411_gb300 import native
    assert native.FEMPIC_ERR_BOUNDS == 10 and native.ERROR_NAMES[10] == "ERR_BOUNDS"
    hdr = open(os.path.join(ROOT, "include", "fempic.h")).read()
    assert "FEMPIC_ERR_BOUNDS = 10" in hdr
