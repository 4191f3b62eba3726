"""Host-side checks of bench.py (no GPU): the traffic figures it reports are tied to the source
text of the streaming-stage kernels, and its reference arm and argument surface are in place."""
import importlib.util
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_stage_kernel_markers_delimit_each_kernel(bench):
    for v, rec in bench.STAGE_KERNELS.items():
        name, begin, end = rec[:3]
        if begin is None or end is None:
            continue
        fname = rec[3] if len(rec) > 3 else "device.cuh"
        src = open(os.path.join(ROOT, "paper_2508_04484_gb300", "csrc", fname)).read()
        i = src.find(begin)
        j = src.find(end, i + 1)
        assert 0 <= i < j, name
        # the delimited text is that kernel's definition and no other stage kernel's
        text = src[i:j]
        assert f"{name}(" in text
        others = [r[0] for w, r in bench.STAGE_KERNELS.items() if w != v and r[0] != name]
        assert not any(f" {o}(" in text for o in others), name
        assert bench.stage_source_sha256(v) is not None


def test_traffic_record_matches_the_current_sources(bench):
    path = os.path.join(ROOT, "profiles", "kstage_traffic.json")
    names = {}
    for v, rec in bench.STAGE_KERNELS.items():
        names.setdefault(rec[0], v)
    for workload, wrec in json.load(open(path))["workloads"].items():
        assert workload in bench.WORKLOADS
        for name, rec in wrec["kernels"].items():
            assert name in names
            assert rec["dram_bytes_per_launch"] == rec["dram_read"] + rec["dram_write"]
            assert "ncu" in rec["capture"] and "--clock-control none" in rec["capture"]
            # the committed figure is reported only while the kernel's text is unchanged
            traffic, note = bench._stage_traffic(names[name], workload)
            if rec["source_sha256"] == bench.stage_source_sha256(names[name]):
                assert traffic == rec["dram_bytes_per_launch"]
            else:
                assert traffic is None and note == "kernel changed since the capture"


def test_stage_work_counts(bench):
    # (5r + 1) words and 2 nk r^2 + 6 nk r flops per cell and launch, four launches per sub-step,
    # none before the first source step (rank 0)
    import numpy as np
    cfg = dict(nx=4, ny=3, nz=2, dy=0.2, precision=1)
    r_start = np.array([0, 2, 3])
    nsub = [5, 2, 1]
    nl, byts, flops = bench.stage_work(cfg, r_start, nsub)
    assert nl == 4 * 2 + 4 * 1
    assert byts == 24 * 4 * (8 * 11 + 4 * 16)
    assert flops == 24 * (8 * (2 * 6 * 4 + 6 * 6 * 2) + 4 * (2 * 6 * 9 + 6 * 6 * 3))
    assert bench._start_ranks(np.array([[-1, 2], [3, 3], [4, -1]])).tolist() == [0, 2, 3]


def test_stage_names_cover_the_autotuner_report(bench):
    # the names dlra_autotune's report uses for the stage variants (paper_2508_04484_gb300/dlra.py)
    from paper_2508_04484_gb300 import dlra as D
    import inspect
    src = inspect.getsource(D.dlra_autotune)
    for name in bench.STAGE_NAMES:
        assert f'"{name}"' in src
    assert sorted(bench.STAGE_NAMES.values()) == sorted(bench.STAGE_KERNELS)
