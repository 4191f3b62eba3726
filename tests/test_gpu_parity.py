"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: the FP64 path must match within 1e-5 relative L2 on the dose, the
FP32-mixed path within 1e-3 (the targets of the build). Low-rank runs replay the
oracle's rank schedule (SCHEDULE mode) so both sides truncate to the same ranks.
Beams are off-centre and tilted: a mirror-symmetric low-rank solution is unstable
to round-off (see tests/test_oracle_solvers.py::test_mirror_symmetry_2d), which
would make any two implementations differ at the truncation level.
"""
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


def _slab(nx=20, nz=24, N=5, collision=WL.BOLTZMANN, n_steps=12, e_max=60.0, e_min=20.0, rank=6, rank_max=8,
          precision=WL.FP64, t100=2e-2, dx=0.2):
    cfg = WL.base_config(nx=nx, ny=1, nz=nz, dx=dx, dy=0.0, dz=dx, N=N, collision=collision,
                         rank_mode=WL.FIXED, rank=rank, rank_max=rank_max, e_max=e_max, e_min=e_min,
                         n_steps=n_steps, precision=precision, t100=t100)
    mats, w = WL.homogeneous(cfg)
    beams = [WL.pencil_beam(e_max, (0.43 * nx * dx, 0.0, 0.0), (0.2, 0.0, 1.0), spot_sigma=0.3)]
    return cfg, mats, w, beams


def _cube(n=10, N=3, n_steps=8, precision=WL.FP32_MIXED, seed=11, rank_mode=WL.ADAPTIVE, rank=8, rank_max=12):
    cfg = WL.base_config(nx=n, ny=n, nz=n, dx=0.25, dy=0.25, dz=0.25, N=N, collision=WL.BOLTZMANN,
                         rank_mode=rank_mode, rank=rank, rank_max=rank_max, trunc_tol=1e-3, e_max=60.0, e_min=30.0,
                         n_steps=n_steps, precision=precision, t100=2e-2)
    mats, w = WL.ellipsoid_phantom(cfg, seed, n_incl=4, semi=(0.3, 0.9))
    beams = [WL.pencil_beam(60.0, (0.47 * n * 0.25, 0.41 * n * 0.25, 0.0), (0.15, -0.1, 1.0), spot_sigma=0.3)]
    return cfg, mats, w, beams


def test_angular_tables_match_oracle():
    cfg, mats, w, beams = _slab(N=7)
    prob = oracle_problem(cfg, mats, w)
    s = gpu_solver(cfg, mats, w, [])
    A, absA = s.tables()
    for d in range(3):
        assert np.abs(A[d] - prob.ang.A[d]).max() < 1e-12
        assert np.abs(absA[d] - (prob.ang.Ap[d] - prob.ang.Am[d])).max() < 1e-12
    assert np.array_equal(s.substeps(), [prob.n_sub(k) for k in range(prob.K)])
    s.close()


@pytest.mark.parametrize("case", ["slab_fp", "cube_boltzmann_spread"])
def test_raytrace_matches_oracle(case):
    if case == "slab_fp":
        cfg, mats, w, beams = _slab(collision=WL.FP, n_steps=20, e_max=60.0, e_min=1.0)
    else:
        cfg, mats, w, beams = _cube(n=8, n_steps=16)
        cfg["e_min"] = 1.0
        beams[0]["energy"] = 50.0
        beams[0]["energy_sigma"] = 1.0
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)[0]
    s = gpu_solver(cfg, mats, w, beams)
    for k in range(prob.K):
        psi, e_u = s.source(k)
        assert rel_l2(psi, src[0][k]) < 1e-8 or np.abs(src[0][k]).max() == 0.0, k
    assert rel_l2(e_u, src[1]) < 1e-8
    s.close()


@pytest.mark.parametrize("precision,tol", [(WL.FP64, 1e-9), (WL.FP32_MIXED, 1e-4)])
def test_one_energy_step_from_a_state(precision, tol):
    cfg, mats, w, beams = _slab(nx=10, nz=12, N=3, n_steps=4, precision=precision)
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    rng = np.random.default_rng(7)
    r = 4
    X, _ = np.linalg.qr(rng.standard_normal((prob.n, r)))
    W, _ = np.linalg.qr(rng.standard_normal((prob.m, r)))
    S = np.diag([1.0, 0.3, 0.1, 0.03]) @ np.linalg.qr(rng.standard_normal((r, r)))[0]
    st = ODL.State(prob.n, prob.m)
    st.X, st.S, st.W = X.copy(), S.copy(), W.copy()
    log = []
    ODL.step(prob, st, 0, src, ODL.RankControl(mode=OP.FIXED, rank=6), log=log)
    sched = np.full((prob.K, 2), -1, dtype=np.int32)
    sched[0] = log[0]
    s = gpu_solver(cfg, mats, w, beams, schedule=sched, precision=precision)
    s.set_state(X, S, W)
    s.step(1)
    Xg, Sg, Wg = s.get_state()
    assert Xg.shape[1] == st.r
    ug = Xg @ Sg @ Wg.T
    assert rel_l2(ug, st.u()) < tol
    s.close()


@pytest.mark.parametrize("precision,tol", [(WL.FP64, 1e-5), (WL.FP32_MIXED, 1e-3), (WL.FP32_SPLIT, 1e-3)])
def test_slab_run_matches_oracle(precision, tol):
    cfg, mats, w, beams = _slab(precision=precision)
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    dose, res = oracle_dlra(prob, src, OP.FIXED, rank=6)
    s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=precision)
    dg = s.run()
    assert np.array_equal(s.rank_log(), res[0]["ranks"])
    assert rel_l2(dg, dose) < tol
    s.close()


@pytest.mark.parametrize("precision,tol", [(WL.FP64, 1e-5), (WL.FP32_MIXED, 1e-3)])
def test_rewound_solve_matches_oracle(precision, tol):
    # a solve after dlra_reset (how the bench repeats solves) must equal the first one
    cfg, mats, w, beams = _slab(precision=precision)
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    dose, res = oracle_dlra(prob, src, OP.FIXED, rank=6)
    s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=precision)
    d1 = s.run()
    s.reset(retrace=True)
    d2 = s.run()
    assert rel_l2(d2, d1) < (1e-12 if precision == WL.FP64 else 1e-5)
    assert rel_l2(d2, dose) < tol
    s.close()


@pytest.mark.parametrize("precision", [WL.FP32_MIXED, WL.FP32_SPLIT])
def test_heterogeneous_cube_fp32_matches_oracle(precision):
    # FP32 stencil and contractions; the truncation SVD and S-step in FP32 (mixed) or FP64 (split)
    cfg, mats, w, beams = _cube()
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    dose, res = oracle_dlra(prob, src, OP.ADAPTIVE, tol=1e-3, r_max=12)
    s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=precision)
    dg = s.run()
    print("precision", precision, "dose error against the FP64 oracle", rel_l2(dg, dose))
    assert rel_l2(dg, dose) < 1e-3
    s.close()


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("case", ["slab", "cube"])
def test_stage_kernel_variants_match_oracle(case, variant):
    # the tcgen05 (3xTF32), the brick-staged and the cell-pair streaming stages against the
    # per-cell stage and the oracle
    if case == "slab":
        cfg, mats, w, beams = _slab(precision=WL.FP32_MIXED)
        mode, kw = OP.FIXED, dict(rank=6)
    else:
        cfg, mats, w, beams = _cube()
        mode, kw = OP.ADAPTIVE, dict(tol=1e-3, r_max=12)
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    dose, res = oracle_dlra(prob, src, mode, **kw)
    doses = []
    for v in (0, variant):
        s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=WL.FP32_MIXED)
        s.set_stage_kernel(v)
        doses.append(s.run())
        s.close()
    assert rel_l2(doses[1], doses[0]) < 1e-5
    assert rel_l2(doses[1], dose) < 1e-3


@pytest.mark.parametrize("case", ["slab", "cube"])
def test_tensor_core_stencil_gram_matches_oracle(case):
    # the L-step and S-step Galerkin blocks on the tensor cores, in a whole solve
    if case == "slab":
        cfg, mats, w, beams = _slab(precision=WL.FP32_MIXED)
        mode, kw = OP.FIXED, dict(rank=6)
    else:
        cfg, mats, w, beams = _cube()
        mode, kw = OP.ADAPTIVE, dict(tol=1e-3, r_max=12)
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    dose, res = oracle_dlra(prob, src, mode, **kw)
    doses = []
    for v in (0, 1):
        s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=WL.FP32_MIXED)
        s.set_stencil_gram_kernel(v)
        doses.append(s.run())
        s.close()
    assert rel_l2(doses[1], doses[0]) < 1e-5
    assert rel_l2(doses[1], dose) < 1e-3


def test_brick_stage_fp64_matches_oracle():
    cfg, mats, w, beams = _slab(precision=WL.FP64)
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    dose, res = oracle_dlra(prob, src, OP.FIXED, rank=6)
    s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=WL.FP64)
    s.set_stage_kernel(2)
    assert rel_l2(s.run(), dose) < 1e-5
    s.close()


def test_state_errors():
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, beams = _slab()
    s = D.Solver(cfg)
    with pytest.raises(D.DlraError) as e:
        s.add_beam(beams[0])
    assert e.value.status == 2
    s.set_materials(mats, w)
    with pytest.raises(D.DlraError) as e:
        s.step(1)
    assert e.value.status == 2
    bad = dict(beams[0], energy=cfg["e_max"] + 5.0)
    with pytest.raises(D.DlraError) as e:
        s.add_beam(bad)
    assert e.value.status == 1
    s.add_beam(beams[0])
    with pytest.raises(D.DlraError) as e:
        s.step(cfg["n_steps"] + 1)
    assert e.value.status == 2
    s.close()


@pytest.mark.parametrize("precision,tol", [(WL.FP64, 1e-5), (WL.FP32_MIXED, 1e-3)])
def test_fokker_planck_delta_correction_matches_oracle(precision, tol):
    # the delta-function corrected Fokker-Planck moments (transport_correction = 2): the
    # uncollided beam is removed at Sigma_t = (xi_1/2)(N+1)(N+2) and feeds a first-collision
    # source with a non-zero l = 0 moment; ray trace and whole solve against the oracle
    cfg, mats, w, beams = _slab(collision=WL.FP, precision=precision)
    cfg["transport_correction"] = 2
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    assert np.abs(src[0][0]).max() > 0
    dose, res = oracle_dlra(prob, src, OP.FIXED, rank=6)
    s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=precision)
    for k in (0, 3, 7):
        psi, e_u = s.source(k)
        assert rel_l2(psi, src[0][0][k]) < 1e-8
    assert rel_l2(e_u, src[0][1]) < 1e-8
    dg = s.run()
    assert np.array_equal(s.rank_log(), res[0]["ranks"])
    err = rel_l2(dg, dose)
    print(f"Fokker-Planck with the delta-function correction, precision {precision}: dose error {err:.2e}")
    assert err < tol
    s.close()
