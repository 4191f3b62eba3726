"""The library's straggling ray trace (csrc/straggling.cu: host preparation of rays, segments and
tables, and the per-ray Crank-Nicolson march of straggling_march.cuh) built as a host program
(tests/straggling_host_march.cu) and run on the CPU, against the oracle's energy-DG tracer
(oracle/straggling.py trace_straggling). Same discretisation, so they agree to FP64 round-off.
Needs nvcc (no GPU)."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import problem as OP
from oracle import straggling as ST
from paper_2508_04484_gb300 import workloads as WL

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2508_04484_gb300", "csrc")


@pytest.fixture(scope="module")
def harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp(prefix="strag_host_")
    exe = os.path.join(d, "march")
    cmd = [nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, "-o", exe, os.path.join(HERE, "straggling_host_march.cu"),
           os.path.join(CSRC, "straggling_tables.cpp"), os.path.join(CSRC, "tables.cpp")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield d, exe
    shutil.rmtree(d, ignore_errors=True)


def _run(harness, cfg, mats, w, beam, G, straggling):
    d, exe = harness
    prob = OP.Problem(cfg, mats, w)
    f = np.zeros(prob.n)
    for i, m in enumerate(prob.phys.mats):
        f += prob.w[i] * m.density * m.sp_ratio
    E = 50.0
    tau = sum(prob.w[i] * prob.phys.sigma_t(i, E) for i in range(prob.M)) / (0.5 * cfg["t100"] * (100.0 / E) ** 2)
    args = [cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"], cfg["e_min"], cfg["e_max"],
            cfg["n_steps"], G, 0.01, cfg["bk_p"], cfg["bk_alpha"], cfg["t100"], int(straggling), beam["energy"],
            beam["energy_sigma"], beam["spot_sigma"], *beam["pos"], *beam["dir"]]
    a_path, c_path, o_path = (os.path.join(d, x) for x in ("args.txt", "cells.bin", "out.bin"))
    with open(a_path, "w") as fh:
        fh.write(" ".join(repr(float(x)) if isinstance(x, float) else str(x) for x in args))
    with open(c_path, "wb") as fh:
        fh.write(np.asarray(f, np.float64).tobytes())
        fh.write(np.asarray(tau, np.float64).tobytes())
    r = subprocess.run([exe, a_path, c_path, o_path], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(o_path, dtype=np.float64)
    K, n = cfg["n_steps"], prob.n
    ref = ST.trace_straggling(prob, beam, n_elem=G, h_max=0.01, straggling=straggling)
    return raw[:K * n].reshape(K, n), raw[K * n:], ref


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("straggling", [False, True])
@pytest.mark.parametrize("spot,esig", [(0.0, 0.0), (0.1, 1.5)])
def test_slab(harness, straggling, spot, esig):
    cfg = WL.base_config(nx=16, ny=1, nz=20, dx=0.2, dy=0.0, dz=0.2, N=3, collision=WL.BOLTZMANN,
                         e_max=66.0, e_min=30.0, n_steps=8, precision=WL.FP64, t100=2e-2)
    mats, w = WL.homogeneous(cfg)
    beam = WL.pencil_beam(60.0, (1.3, 0.0, 0.0), (0.2, 0.0, 1.0), spot_sigma=spot, energy_sigma=esig)
    psi, e_u, ref = _run(harness, cfg, mats, w, beam, 128, straggling)
    assert _rel(e_u, ref.e_u) < 1e-12 and _rel(psi, ref.psi) < 1e-12


def test_heterogeneous_cube(harness):
    cfg = WL.base_config(nx=8, ny=7, nz=10, dx=0.25, dy=0.25, dz=0.25, N=3, collision=WL.BOLTZMANN,
                         e_max=62.0, e_min=30.0, n_steps=6, precision=WL.FP64, t100=2e-2)
    mats, w = WL.ellipsoid_phantom(cfg, 5, n_incl=3, semi=(0.3, 0.8))
    beam = WL.pencil_beam(58.0, (1.0, 0.9, 0.0), (0.15, -0.1, 1.0), spot_sigma=0.15, energy_sigma=1.0)
    psi, e_u, ref = _run(harness, cfg, mats, w, beam, 64, True)
    assert _rel(e_u, ref.e_u) < 1e-12 and _rel(psi, ref.psi) < 1e-12
