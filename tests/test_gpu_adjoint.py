"""Reverse sweep (dlra_backward) against the oracle.

With one energy step the low-rank solve is exact (the source step from rank 0 spans the
source exactly) and the GPU gradient equals the full-rank discrete adjoint
(oracle/adjoint.py). Over several steps the GPU runs the low-rank reverse sweep, which is
compared at round-off with its plain restatement (oracle/dlra_adjoint.py) and within the
approximation level with the full-rank gradient.
"""
import numpy as np
import pytest

from oracle import adjoint as OAD
from oracle import problem as OP
from paper_2508_04484_gb300 import workloads as WL

from .gpu_util import rel_l2

pytestmark = pytest.mark.gpu

WATER = dict(density=1.0, sp_ratio=1.0, scatter_ratio=1.0, screening=1e-3)
BONE = dict(density=1.85, sp_ratio=0.9, scatter_ratio=1.35, screening=1.5e-3)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    build.build()


def _case(nx=6, nz=6, N=3, K=1, collision=WL.BOLTZMANN, rank_mode=WL.FIXED, rank=8, rank_max=8, tol=1e-3,
          precision=WL.FP64, seed=1, t100=1e-2):
    cfg = WL.base_config(nx=nx, ny=1, nz=nz, dx=0.25, dy=0.0, dz=0.25, N=N, collision=collision,
                         rank_mode=rank_mode, rank=rank, rank_max=rank_max, trunc_tol=tol, e_max=60.0,
                         e_min=40.0, n_steps=K, precision=precision, t100=t100)
    rng = np.random.default_rng(seed)
    n = nx * nz
    w = rng.uniform(0.2, 1.0, (2, n))
    w /= w.sum(0)
    g = rng.standard_normal(n)
    return cfg, [WATER, BONE], w, g


def _gpu_grad(cfg, mats, w, beams, g, interval=16, keep=True, stage=None):
    from paper_2508_04484_gb300 import dlra as D
    s = D.Solver(cfg, mats, w, beams)
    s.set_adjoint_store(keep)
    if stage is not None:
        s.set_stage_kernel(stage)
    s.enable_adjoint(interval)
    e = s.run()
    dbeta, dw = s.backward(g)
    s.close()
    return e, dbeta, dw


def _oracle_grad(cfg, mats, w, beams, g):
    prob = OP.Problem(cfg, mats, w)
    e = OAD.loss_and_dose(prob, beams)
    return e, OAD.gradient(prob, beams, g)


PENCILS = [WL.pencil_beam(60.0, (0.7, 0.0, 0.0), (0.3, 0.0, 1.0), spot_sigma=0.0, weight=0.8),
           WL.pencil_beam(55.0, (1.0, 0.0, 0.0), (-0.2, 0.0, 1.0), spot_sigma=0.1, weight=1.3)]


@pytest.mark.parametrize("collision", [WL.BOLTZMANN, WL.FP])
def test_one_step_gradient_matches_oracle(collision):
    cfg, mats, w, g = _case(collision=collision)
    e, dbeta, dw = _gpu_grad(cfg, mats, w, PENCILS, g)
    eo, go = _oracle_grad(cfg, mats, w, PENCILS, g)
    print("dose", rel_l2(e, eo), "dbeta", rel_l2(dbeta, go["dbeta"]), "dw", rel_l2(dw, go["dw"]),
          "dw_trace share", np.linalg.norm(go["dw_trace"]) / np.linalg.norm(go["dw"]))
    assert rel_l2(e, eo) < 1e-7
    assert rel_l2(dbeta, go["dbeta"]) < 1e-7
    assert rel_l2(dw, go["dw"]) < 1e-5


def _multi_case(precision=WL.FP64, K=6, t100=0.1):
    return _case(nx=8, nz=8, N=3, K=K, rank_mode=WL.ADAPTIVE, rank=16, rank_max=16, tol=1e-6,
                 precision=precision, seed=2, t100=t100)


ONE_BEAM = [WL.pencil_beam(60.0, (1.1, 0.0, 0.0), (0.2, 0.0, 1.0), spot_sigma=0.1, weight=1.0)]


def _low_rank_oracle(cfg, mats, w, beams, g):
    from oracle import dlra as ODL
    from oracle import dlra_adjoint as OLA
    rc = ODL.RankControl(mode=cfg["rank_mode"], rank=cfg["rank"], tol=cfg["trunc_tol"], r_max=cfg["rank_max"])
    return OLA.gradient(OP.Problem(cfg, mats, w), beams, g, rc)


@pytest.mark.parametrize("smooth", [False, True])
def test_multi_step_gradient_matches_low_rank_oracle_fp64(smooth):
    cfg, mats, w, g = _multi_case()
    if smooth:
        x = (np.arange(8) + 0.5) * 0.25
        Xg, Zg = np.meshgrid(x, x)
        g = np.exp(-((Xg - 1.2) ** 2 + (Zg - 1.0) ** 2) / 0.5).ravel()
    e, dbeta, dw = _gpu_grad(cfg, mats, w, ONE_BEAM, g)
    lo = _low_rank_oracle(cfg, mats, w, ONE_BEAM, g)
    print("vs low-rank oracle: dbeta", rel_l2(dbeta, lo["dbeta"]), "dw", rel_l2(dw, lo["dw"]))
    assert rel_l2(dbeta, lo["dbeta"]) < 1e-9
    assert rel_l2(dw, lo["dw"]) < 1e-8


def test_multi_step_gradient_fp32_mixed_matches_low_rank_oracle():
    # a smooth dL/de: a random-sign one makes <dL/de, e_b> a cancelling sum
    cfg, mats, w, g = _multi_case(WL.FP32_MIXED)
    x = (np.arange(8) + 0.5) * 0.25
    Xg, Zg = np.meshgrid(x, x)
    g = np.exp(-((Xg - 1.2) ** 2 + (Zg - 1.0) ** 2) / 0.5).ravel()
    e, dbeta, dw = _gpu_grad(cfg, mats, w, ONE_BEAM, g)
    cfg64 = dict(cfg, precision=WL.FP64)
    lo = _low_rank_oracle(cfg64, mats, w, ONE_BEAM, g)
    print("fp32 vs low-rank oracle: dbeta", rel_l2(dbeta, lo["dbeta"]), "dw", rel_l2(dw, lo["dw"]))
    assert rel_l2(dbeta, lo["dbeta"]) < 2e-3
    assert rel_l2(dw, lo["dw"]) < 5e-3


def test_gradient_is_within_truncation_level_of_full_rank():
    # energy steps of 0.83 MeV on 2.5 mm cells (the bench workload: 0.745 MeV on 2 mm)
    cfg, mats, w, g = _multi_case(K=24, t100=1e-2)
    e, dbeta, dw = _gpu_grad(cfg, mats, w, ONE_BEAM, g)
    eo, go = _oracle_grad(cfg, mats, w, ONE_BEAM, g)
    print("vs full rank: dose", rel_l2(e, eo), "dbeta", rel_l2(dbeta, go["dbeta"]), "dw", rel_l2(dw, go["dw"]))
    assert rel_l2(e, eo) < 1e-3
    assert rel_l2(dbeta, go["dbeta"]) < 1e-3
    assert rel_l2(dw, go["dw"]) < 1.5e-2


def test_checkpoint_interval_does_not_change_the_gradient():
    cfg, mats, w, g = _multi_case()
    beams = [WL.pencil_beam(60.0, (1.1, 0.0, 0.0), (0.2, 0.0, 1.0), spot_sigma=0.1, weight=1.0),
             WL.pencil_beam(57.0, (0.9, 0.0, 0.0), (-0.1, 0.0, 1.0), spot_sigma=0.1, weight=0.5)]
    out = [_gpu_grad(cfg, mats, w, beams, g, interval=I) for I in (1, 4, 16)]
    for e, dbeta, dw in out[1:]:
        print("interval", rel_l2(dw, out[0][2]), rel_l2(dbeta, out[0][1]))
        assert rel_l2(e, out[0][0]) < 1e-12
        assert rel_l2(dbeta, out[0][1]) < 1e-12
        assert rel_l2(dw, out[0][2]) < 1e-9


def test_kept_and_recomputed_forward_steps_agree():
    """The reverse sweep with the replayed stage inputs kept, and with them recomputed."""
    cfg, mats, w, g = _multi_case()
    beams = [WL.pencil_beam(60.0, (1.1, 0.0, 0.0), (0.2, 0.0, 1.0), spot_sigma=0.1, weight=1.0),
             WL.pencil_beam(57.0, (0.9, 0.0, 0.0), (-0.1, 0.0, 1.0), spot_sigma=0.1, weight=0.5)]
    for interval in (3, 16):
        kept = _gpu_grad(cfg, mats, w, beams, g, interval=interval, keep=True)
        redo = _gpu_grad(cfg, mats, w, beams, g, interval=interval, keep=False)
        assert rel_l2(kept[1], redo[1]) < 1e-12
        assert rel_l2(kept[2], redo[2]) < 1e-9


@pytest.mark.parametrize("stage", [2, 3])
def test_stage_kernel_variants_give_the_same_gradient(stage):
    # the transposed streaming stage of the reverse sweep in the brick and cell-pair kernels
    # fixed rank: the variants differ in the last bit, which must not flip an adaptive rank decision
    cfg, mats, w, _ = _case(nx=8, nz=8, N=3, K=6, rank_mode=WL.FIXED, rank=8, rank_max=16,
                            precision=WL.FP32_MIXED, seed=2, t100=0.1)
    n = cfg["nx"] * cfg["nz"]
    g = np.sin(np.arange(n) * 0.37) + 1.5
    e0, b0, w0 = _gpu_grad(cfg, mats, w, ONE_BEAM, g, stage=0)
    e1, b1, w1 = _gpu_grad(cfg, mats, w, ONE_BEAM, g, stage=stage)
    assert rel_l2(e1, e0) < 1e-5
    assert rel_l2(b1, b0) < 1e-4
    assert rel_l2(w1, w0) < 1e-3


def test_beam_weights_and_mixture_replacement():
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, g = _case(K=3, seed=4)
    beams = [dict(b) for b in PENCILS]
    s = D.Solver(cfg, mats, w, beams)
    s.enable_adjoint(2)
    e1 = s.run()
    # a new weight changes the dose linearly without stepping again
    s.set_beam_weight(1, 0.0)
    e0 = s.dose()
    s.set_beam_weight(1, 2.6)
    e2 = s.dose()
    assert rel_l2(e2 - e0, 2.0 * (e1 - e0)) < 1e-12
    # weight 0 still has the unit-weight gradient <dL/de, e_b>
    s.set_beam_weight(1, 0.0)
    dbeta, _ = s.backward(g)
    assert abs(dbeta[1] - g @ ((e1 - e0) / 1.3)) < 1e-10 * abs(dbeta[1])
    # replacing the mixture retraces and rewinds; the result equals a fresh solver
    rng = np.random.default_rng(9)
    w2 = rng.uniform(0.2, 1.0, w.shape)
    w2 /= w2.sum(0)
    s.set_beam_weight(1, 1.3)
    s.set_materials(mats, w2)
    assert s.query()[0] == 0
    e3 = s.run()
    s.close()
    f = D.Solver(cfg, mats, w2, beams)
    e4 = f.run()
    f.close()
    assert rel_l2(e3, e4) < 1e-12


def test_autograd_function():
    import torch
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, g = _case(K=2, seed=5)
    s = D.Solver(cfg, mats, w, PENCILS)
    s.enable_adjoint(16)
    wt = torch.tensor(w, dtype=torch.float64, device="cuda", requires_grad=True)
    bt = torch.tensor([0.8, 1.3], dtype=torch.float64, requires_grad=True)
    e = D.differentiable_dose(s, mats, wt, bt)
    gt = torch.tensor(g, dtype=torch.float64, device="cuda")
    loss = (gt * e).sum()
    loss.backward()
    dbeta, dw = s.backward(g)
    assert torch.allclose(wt.grad.cpu(), torch.tensor(dw), rtol=1e-12, atol=0)
    assert np.allclose(bt.grad.numpy(), dbeta, rtol=1e-12, atol=0)
    s.close()


def test_backward_call_order():
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, g = _case(K=2)
    s = D.Solver(cfg, mats, w, PENCILS[:1])
    with pytest.raises(D.DlraError) as ex:
        s.backward(g)
    assert ex.value.status == D.DLRA_ERR_STATE
    s.step(1)
    with pytest.raises(D.DlraError) as ex:
        s.enable_adjoint(4)
    assert ex.value.status == D.DLRA_ERR_STATE
    s.reset()
    s.enable_adjoint(4)
    s.step(2)
    dbeta, dw = s.backward(np.zeros_like(g))
    assert np.all(dbeta == 0) and np.all(dw == 0)
    s.close()
