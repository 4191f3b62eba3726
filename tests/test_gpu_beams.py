"""Several beams in one context: independent low-rank states advanced concurrently
(one lane per beam) or one after the other give the same dose, equal to the sum
of the oracle's single-beam solves."""
import numpy as np
import pytest

from oracle import problem as OP
from paper_2508_04484_gb300 import workloads as WL

from .gpu_util import oracle_dlra, oracle_problem, oracle_sources, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    build.build()


def _case():
    cfg = WL.base_config(nx=20, ny=1, nz=22, dx=0.2, dy=0.0, dz=0.2, N=5, collision=WL.BOLTZMANN,
                         rank_mode=WL.FIXED, rank=6, rank_max=8, e_max=60.0, e_min=25.0, n_steps=10,
                         precision=WL.FP64, t100=2e-2)
    mats, w = WL.homogeneous(cfg)
    beams = [WL.pencil_beam(60.0, (1.7, 0.0, 0.0), (0.2, 0.0, 1.0), weight=1.0),
             WL.pencil_beam(55.0, (2.4, 0.0, 0.0), (-0.15, 0.0, 1.0), weight=0.7),
             WL.pencil_beam(50.0, (1.3, 0.0, 0.0), (0.05, 0.0, 1.0), weight=1.3)]
    return cfg, mats, w, beams


def test_concurrent_beams_match_sequential_and_oracle():
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, beams = _case()
    doses = []
    for lanes in (1, 3):
        s = D.Solver(dict(cfg, max_concurrent_beams=lanes), mats, w, beams)
        doses.append(s.run())
        logs = [s.rank_log(b) for b in range(3)]
        s.close()
    assert rel_l2(doses[1], doses[0]) < 1e-12
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    ref, res = oracle_dlra(prob, src, OP.FIXED, rank=6)
    for b in range(3):
        assert np.array_equal(logs[b], res[b]["ranks"]), b
    assert rel_l2(doses[1], ref) < 1e-5


def test_graph_replay_matches_direct_launches():
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, beams = _case()
    s = D.Solver(dict(cfg, max_concurrent_beams=3), mats, w, beams)
    ref = s.run()
    l_direct = s.launch_count()
    s.set_graphs(True)
    for _ in range(3):                       # capture on the first pass, replay afterwards
        s.reset(retrace=True)
        d = s.run()
        assert rel_l2(d, ref) < 1e-12
    assert s.launch_count() > 3 * l_direct // 2    # replays count the kernels they contain
    # split solves are separate graphs; profiling bypasses them
    s.reset(retrace=True)
    s.step(4)
    s.set_profiling(True)
    s.step(3)
    s.set_profiling(False)
    s.step(cfg["n_steps"] - 7)
    assert rel_l2(s.dose(), ref) < 1e-12
    s.set_graphs(False)
    s.close()


def test_autotuned_launches_give_the_same_dose():
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, beams = _case()
    cfg = dict(cfg, precision=WL.FP32_MIXED)
    s = D.Solver(cfg, mats, w, beams)
    ref = s.run()
    rep = s.autotune()
    assert rep["stage_fma_ms"] > 0 and rep["stage_tensor_core_ms"] > 0 and rep["stage_brick_ms"] > 0
    assert rep["gram_blocks"] in (608, 1216, 2432, 4864)
    s.reset(retrace=True)
    d = s.run()
    assert rel_l2(d, ref) < 1e-5
    s.close()
