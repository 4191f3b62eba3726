"""GPU parity of the joint multi-beam state (dlra_set_joint; the paper's multi-beam solve, Sec. 4.3):
all beams feed one low-rank state. The oracle's low-rank solve given several sources is that
joint solve (oracle/dlra.py, step: the active sources' factors are stacked into one source).
Two near-perpendicular beams on a water slab, weights 0.7 and 1.3, the oracle's rank schedule
replayed; FP64 within 1e-5 and FP32 within 1e-3 of the oracle's dose."""
import numpy as np
import pytest

from oracle import dlra as ODL
from oracle import problem as OP
from paper_2508_04484_gb300 import workloads as WL

from .gpu_util import gpu_solver, oracle_dlra, oracle_problem, oracle_sources, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    build.build()


def _case(precision):
    cfg = WL.base_config(nx=24, ny=1, nz=24, dx=0.1, dy=0.0, dz=0.1, N=5, collision=WL.BOLTZMANN,
                         rank_mode=WL.ADAPTIVE, rank=24, rank_max=24, trunc_tol=1e-3, e_max=50.0, e_min=20.0,
                         n_steps=12, precision=precision, t100=2e-2)
    mats, w = WL.homogeneous(cfg)
    beams = [WL.pencil_beam(50.0, (1.07, 0.0, 0.0), (0.08, 0.0, 1.0), spot_sigma=0.2, weight=0.7),
             WL.pencil_beam(48.0, (0.0, 0.0, 1.31), (1.0, 0.0, 0.06), spot_sigma=0.2, weight=1.3)]
    return cfg, mats, w, beams


@pytest.mark.parametrize("precision,tol", [(WL.FP64, 1e-5), (WL.FP32_MIXED, 1e-3)])
def test_joint_state_matches_oracle(precision, tol):
    cfg, mats, w, beams = _case(precision)
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)           # weighted beams: the tracer carries the weight
    joint = ODL.solve(prob, src, ODL.RankControl(mode=OP.ADAPTIVE, tol=1e-3, r_max=24))
    s = gpu_solver(cfg, mats, w, beams, schedule=joint["ranks"], precision=precision)
    s.set_joint(True)
    dg = s.run()
    assert np.array_equal(s.rank_log(0), joint["ranks"])
    err = rel_l2(dg, joint["dose"])
    _, indep = oracle_dlra(prob, src, OP.ADAPTIVE, tol=1e-3, r_max=24)
    r_joint = int(joint["ranks"][-1][1] if joint["ranks"][-1][1] >= 0 else joint["ranks"][-1][0])
    r_each = [int(r["ranks"][-1][1] if r["ranks"][-1][1] >= 0 else r["ranks"][-1][0]) for r in indep]
    print(f"joint state, precision {precision}: dose error {err:.2e}; final rank {r_joint} (each beam alone {r_each})")
    assert err < tol
    s.close()


def test_joint_mode_refuses_the_reverse_sweep():
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, beams = _case(WL.FP64)
    s = gpu_solver(cfg, mats, w, beams)
    s.set_joint(True)
    with pytest.raises(D.DlraError) as e:
        s.enable_adjoint(4)
    assert e.value.status == 2
    s.close()
