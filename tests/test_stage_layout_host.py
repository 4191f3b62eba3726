"""The layout of the tensor-core streaming stages with five TMA boxes per chunk
(csrc/kstage_tmaf.cuh), checked on the CPU before they run on a GPU: tests/stage_layout_host.cu
evaluates the kernel's own offset function for every formation thread, warp group, chunk column
and stencil point and checks that each read lands in the box holding that neighbour, at the
neighbour's position, and that the shared-memory and TMEM budgets, the expected copy bytes and
the TMA alignment rules hold, at every rank capacity the library instantiates. Needs nvcc (no
GPU)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_04484_gb300", "csrc")


def test_five_box_stage_layout():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="stage_layout_")
    try:
        exe = os.path.join(d, "layout")
        cmd = [nvcc, "-O1", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I",
               os.path.join(ROOT, "include"), "-I", CSRC, "-o", exe, os.path.join(HERE, "stage_layout_host.cu")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        lines = r.stdout.strip().splitlines()
        assert len(lines) == 8
        # 2 warp groups x 128 cells x 2 columns x 13 stencil points per configuration
        assert all(line.endswith("6656 reads checked") for line in lines), r.stdout
    finally:
        shutil.rmtree(d, ignore_errors=True)
