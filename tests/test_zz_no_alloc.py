"""The allocation-free K-step entry point.

Some callers cannot call cudaMalloc: they run inside a memory pool they do not
own, on paths that must not synchronise the device, or in runtimes that only hand
out pre-registered buffers. dlra_kstep_noalloc serves them with a static device
work space; here its output is checked against the allocating dlra_kstep on two
calls in a row (the work space keeps the previous call's contents), and an
oversized problem is rejected on the host with a clear error.
"""
import numpy as np
import pytest

from .gpu_util import rel_l2
from .test_gpu_kstep import kstep_case, run_kstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    from paper_2508_04484_gb300 import dlra as D
    build.build()
    return D


@pytest.mark.parametrize("two_d", [False, True])
def test_noalloc_kstep_matches_allocating_kstep(lib, two_d):
    cfg, prob, X, S, W, k, Pk, rho_s = kstep_case(two_d, seed=5)
    ref = run_kstep(lib.dlra_kstep, cfg, prob, X, S, k, Pk, rho_s)
    for _ in range(2):
        out = run_kstep(lib.dlra_kstep_noalloc, cfg, prob, X, S, k, Pk, rho_s)
        assert rel_l2(out, ref) < 1e-5


def test_noalloc_rejects_work_space_beyond_the_maximum(lib):
    import torch
    dev = torch.device("cuda", 0)
    grid = dict(nx=256, ny=128, nz=128, dx=0.1, dy=0.1, dz=0.1)   # 4.2M cells: > 32 MiB at r = 8
    tiny = torch.zeros(1, dtype=torch.float32, device=dev)
    a = lib.kstep_args(grid, 8, 100.0, 1.0, 1, tiny, torch.zeros(1, dtype=torch.float32, device=dev), tiny, tiny)
    with pytest.raises(lib.DlraError) as e:
        lib.dlra_kstep_noalloc(a)
    assert e.value.status == 1
    assert "static work space" in str(e.value)
