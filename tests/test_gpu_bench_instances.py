"""GPU parity at the kernel instances the measured workloads run, against the FP64 oracle.

* The 2-D x-z slab of 40 x 40 cells of 1 mm (Fokker-Planck, P_7, rank 5, 60 energy steps
  100 -> 1 MeV, FP64) end to end, with the oracle's rank schedule replayed (1e-5).
* The streaming stage, tall-skinny products, moment-side L-step and truncation SVD at the
  widths of the 64^3 water workload (P_15, m = 256, rank 20, 2r = 40; 3-D, six stencils) and
  of the 128^3 phantom workload (P_21, m = 484, rank capacity 64, 2r = 128, three materials):
  a 24^3 grid with the same voxel size, physics and rank capacity, started from a seeded
  full-rank state (random orthonormal factors, decaying singular values) and advanced over a
  few energy steps at the workloads' energy step, both FP32 paths (1e-3 on u = X S W^T and on
  the dose).

Beams are off-centre and tilted (a mirror-symmetric low-rank solution is unstable to round-off:
tests/test_oracle_solvers.py::test_mirror_symmetry_2d); the 40 x 40 slab keeps its
face-centred normal beam, where a 1e-13 change of the input moves the oracle's own dose by 5e-6.
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


@pytest.mark.parametrize("beam", ["tilted", "centred"])
def test_slab_40x40_fokker_planck_end_to_end(beam):
    # the workload's face-centred normal beam is mirror-symmetric: the low-rank solution is then
    # ill-conditioned (in the oracle alone, a 1e-13 change of one mixture weight moves the dose
    # by 5e-6 and a 1e-11 change by 6e-5, while the same changes move the tilted beam's dose by
    # < 1e-15), so two correct implementations agree there only to the truncation level; the
    # same grid, physics, rank and energy steps with an off-centre tilted beam carry the 1e-5 bar
    cfg, mats, w, beams = WL.slab_fp_40x40()
    if beam == "tilted":
        beams = [WL.pencil_beam(100.0, (1.93, 0.0, 0.0), (0.05, 0.0, 1.0))]
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    dose, res = oracle_dlra(prob, src, OP.FIXED, rank=5)
    s = gpu_solver(cfg, mats, w, beams, schedule=res[0]["ranks"], precision=WL.FP64)
    dg = s.run()
    assert np.array_equal(s.rank_log(), res[0]["ranks"])
    err = rel_l2(dg, dose)
    print(f"slab 40x40 FP64, {beam} beam: dose error against the oracle {err:.2e}")
    assert err < (1e-5 if beam == "tilted" else 5e-3)
    s.close()


def _instance(kind, precision):
    """A 24^3 grid with a workload's voxel size, physics, angular degree and rank capacity."""
    if kind == "water_64cube":
        cfg = WL.base_config(nx=24, ny=24, nz=24, dx=0.2, dy=0.2, dz=0.2, N=15, collision=WL.BOLTZMANN,
                             transport_correction=1, rank_mode=WL.FIXED, rank=20, rank_max=20, e_max=150.0,
                             e_min=150.0 - 3 * 0.745, n_steps=3, precision=precision)
        mats, w = WL.homogeneous(cfg)
        beams = [WL.pencil_beam(150.0, (2.27, 2.51, 0.0), (0.12, -0.08, 1.0), spot_sigma=0.1)]
        r, mode, kw = 20, OP.FIXED, dict(rank=20)
    else:
        cfg = WL.base_config(nx=24, ny=24, nz=24, dx=0.15, dy=0.15, dz=0.15, N=21, collision=WL.BOLTZMANN,
                             transport_correction=1, rank_mode=WL.ADAPTIVE, rank=60, rank_max=60, trunc_tol=1e-3,
                             e_max=180.0, e_min=179.0, n_steps=2, precision=precision)
        mats, w = WL.ellipsoid_phantom(cfg, 3, n_incl=5, semi=(0.3, 1.0))
        beams = [WL.pencil_beam(180.0, (1.71, 1.86, 0.0), (0.1, 0.07, 1.0), spot_sigma=0.1)]
        r, mode, kw = 60, OP.ADAPTIVE, dict(tol=1e-3, r_max=60)
    return cfg, mats, w, beams, r, mode, kw


def _state(prob, r, seed):
    rng = np.random.default_rng(seed)
    X, _ = np.linalg.qr(rng.standard_normal((prob.n, r)))
    W, _ = np.linalg.qr(rng.standard_normal((prob.m, r)))
    sig = 1e-2 * 0.85 ** np.arange(r)
    S = np.diag(sig) @ np.linalg.qr(rng.standard_normal((r, r)))[0]
    return X, S, W


_ORACLE = {}


def _oracle_run(kind):
    """The oracle's steps from the seeded state (computed once per workload kind)."""
    if kind not in _ORACLE:
        cfg, mats, w, beams, r, mode, kw = _instance(kind, WL.FP64)
        prob = oracle_problem(cfg, mats, w)
        src = oracle_sources(prob, beams)
        X, S, W = _state(prob, r, 17)
        st = ODL.State(prob.n, prob.m)
        st.X, st.S, st.W = X.copy(), S.copy(), W.copy()
        rc = ODL.RankControl(mode=mode, **kw)
        log = []
        e_c = np.zeros(prob.n)
        for k in range(prob.K):
            ODL.step(prob, st, k, src, rc, log=log)
            e_c += prob.h * np.sqrt(4 * np.pi) * st.moment0()
        _ORACLE[kind] = (prob, src, (X, S, W), st, log, e_c)
    return _ORACLE[kind]


@pytest.mark.parametrize("precision", [WL.FP32_MIXED, WL.FP32_SPLIT])
@pytest.mark.parametrize("kind", ["water_64cube", "phantom_128cube"])
def test_workload_kernel_instances_match_oracle(kind, precision):
    cfg, mats, w, beams, r, mode, kw = _instance(kind, precision)
    prob, src, (X, S, W), st, log, e_c = _oracle_run(kind)
    s = gpu_solver(cfg, mats, w, beams, schedule=np.asarray(log, dtype=np.int32), precision=precision)
    s.set_state(X, S, W)
    s.step(prob.K)
    dg = s.dose()
    Xg, Sg, Wg = s.get_state()
    assert np.array_equal(s.rank_log(), np.asarray(log))
    eu = src[0][1]
    err_u = rel_l2(Xg @ Sg @ Wg.T, st.u())
    err_d = rel_l2(dg - eu, e_c)
    print(f"{kind} precision {precision}: ranks {[tuple(x) for x in log]}, u error {err_u:.2e}, "
          f"collided dose error {err_d:.2e}")
    assert err_u < 1e-3
    assert err_d < 1e-3
    s.close()


@pytest.mark.parametrize("variant", [4, 5, 6, 7, 8, 9, 10, 11, 12, 13])
@pytest.mark.parametrize("case", ["ragged", "phantom_128cube"])
def test_tma_tensor_core_stage_matches_oracle(case, variant):
    # the TMA-staged tensor-core streaming stage (128- and 256-cell bricks) against the per-cell
    # FMA stage and the oracle: on a grid whose bricks are ragged in every direction (rank
    # capacity 40, MMA N = 48) and at the 128^3 phantom workload's widths (capacity 64)
    if case == "ragged":
        cfg, mats, w, beams, prob, (X, S, W), st, log = _ragged_instance()
    else:
        cfg, mats, w, beams, r, mode, kw = _instance(case, WL.FP32_MIXED)
        prob, src, (X, S, W), st, log, _ = _oracle_run(case)
    us = []
    for v in (0, variant):
        s = gpu_solver(cfg, mats, w, beams, schedule=np.asarray(log, dtype=np.int32), precision=WL.FP32_MIXED)
        s.set_stage_kernel(v)
        s.set_state(X, S, W)
        s.step(prob.K)
        Xg, Sg, Wg = s.get_state()
        us.append(Xg @ Sg @ Wg.T)
        s.close()
    e_fma, e_or = rel_l2(us[1], us[0]), rel_l2(us[1], st.u())
    print(f"TMA stage variant {variant} on {case}: against the FMA stage {e_fma:.2e}, against the oracle {e_or:.2e}")
    assert e_fma < KERNEL_BOUND[case]
    assert e_or < 1e-3


# Two FP32 variants of one kernel round differently; over whole energy steps the difference is
# amplified like any other FP32 rounding. Their bound is set against the FP32 path's own distance
# to the oracle on the same instance: 1.4e-5 on the ragged grid (bound 1e-5), 6.5e-5 on the
# phantom instance (bound 3e-5: measured differences 5e-6 .. 1.04e-5 as shared kernels changed
# their summation order).
KERNEL_BOUND = {"ragged": 1e-5, "phantom_128cube": 3e-5}


def _ragged_instance():
    # a grid whose 128-cell tiles and bricks are ragged in every direction (3,600 cells), rank 40
    # (MMA N = 48), advanced by the oracle over two energy steps from a seeded state
    cfg = WL.base_config(nx=20, ny=18, nz=10, dx=0.2, dy=0.2, dz=0.2, N=7, collision=WL.BOLTZMANN,
                         rank_mode=WL.FIXED, rank=40, rank_max=40, e_max=120.0, e_min=118.0, n_steps=2,
                         precision=WL.FP32_MIXED)
    mats, w = WL.ellipsoid_phantom(cfg, 9, n_incl=3, semi=(0.3, 0.9))
    beams = [WL.pencil_beam(120.0, (1.71, 1.53, 0.0), (0.1, 0.07, 1.0), spot_sigma=0.1)]
    prob = oracle_problem(cfg, mats, w)
    src = oracle_sources(prob, beams)
    X, S, W = _state(prob, 40, 23)
    st = ODL.State(prob.n, prob.m)
    st.X, st.S, st.W = X.copy(), S.copy(), W.copy()
    log = []
    for k in range(prob.K):
        ODL.step(prob, st, k, src, ODL.RankControl(mode=OP.FIXED, rank=40), log=log)
    return cfg, mats, w, beams, prob, (X, S, W), st, log


@pytest.mark.parametrize("case", ["ragged", "phantom_128cube"])
def test_tensor_core_apply_matches_oracle(case):
    # the cell-side tall-skinny products on the tensor cores (augmentation projections, the
    # truncation's X = X^ P), forced at every height (kernel 2), on ragged 128-row tiles and at
    # the 128^3 phantom workload's widths: against the FMA products and the oracle
    if case == "ragged":
        cfg, mats, w, beams, prob, (X, S, W), st, log = _ragged_instance()
    else:
        cfg, mats, w, beams, r, mode, kw = _instance(case, WL.FP32_MIXED)
        prob, src, (X, S, W), st, log, _ = _oracle_run(case)
    us = []
    for v in (0, 2):
        s = gpu_solver(cfg, mats, w, beams, schedule=np.asarray(log, dtype=np.int32), precision=WL.FP32_MIXED)
        s.set_apply_kernel(v)
        s.set_state(X, S, W)
        s.step(prob.K)
        Xg, Sg, Wg = s.get_state()
        us.append(Xg @ Sg @ Wg.T)
        s.close()
    e_fma, e_or = rel_l2(us[1], us[0]), rel_l2(us[1], st.u())
    print(f"tensor-core apply on {case}: against the FMA products {e_fma:.2e}, against the oracle {e_or:.2e}")
    # the two kernels round differently: equal results would mean the tensor-core path never ran
    assert 0.0 < e_fma < KERNEL_BOUND[case]
    assert e_or < 1e-3


@pytest.mark.parametrize("case", ["ragged", "phantom_128cube"])
def test_windowed_stencil_gram_in_solver(case):
    # the L-step and S-step Galerkin blocks on the tensor cores with the sliding TMA window
    # (stencil-Gram kernel 2; r x r at capacity 40 / 64 and 2r x 2r at 80 / 128 columns) inside
    # whole energy steps: against the FMA Grams and the oracle
    if case == "ragged":
        cfg, mats, w, beams, prob, (X, S, W), st, log = _ragged_instance()
    else:
        cfg, mats, w, beams, r, mode, kw = _instance(case, WL.FP32_MIXED)
        prob, src, (X, S, W), st, log, _ = _oracle_run(case)
    us = []
    for v in (0, 2):
        s = gpu_solver(cfg, mats, w, beams, schedule=np.asarray(log, dtype=np.int32), precision=WL.FP32_MIXED)
        s.set_stencil_gram_kernel(v)
        s.set_state(X, S, W)
        s.step(prob.K)
        Xg, Sg, Wg = s.get_state()
        us.append(Xg @ Sg @ Wg.T)
        s.close()
    e_fma, e_or = rel_l2(us[1], us[0]), rel_l2(us[1], st.u())
    print(f"windowed stencil Gram on {case}: against the FMA Grams {e_fma:.2e}, against the oracle {e_or:.2e}")
    assert 0.0 < e_fma < KERNEL_BOUND[case]
    assert e_or < 1e-3


@pytest.mark.parametrize("case", ["ragged", "phantom_128cube"])
def test_tensor_core_grams_in_solver(case):
    # the cell-side tall-skinny Grams on the tensor cores, forced at every height (Gram kernel 2):
    # the augmentation's X^T K (B its own array), the CholeskyQR2 Grams (B a column block of X^),
    # the material Grams X^T diag(w_k) X (weighted; at capacity 40 a slice of 64 columns spans
    # two materials), on a ragged last chunk and at the phantom widths: against the FMA Grams
    # and the oracle
    if case == "ragged":
        cfg, mats, w, beams, prob, (X, S, W), st, log = _ragged_instance()
    else:
        cfg, mats, w, beams, r, mode, kw = _instance(case, WL.FP32_MIXED)
        prob, src, (X, S, W), st, log, _ = _oracle_run(case)
    us = []
    for v in (0, 2):
        s = gpu_solver(cfg, mats, w, beams, schedule=np.asarray(log, dtype=np.int32), precision=WL.FP32_MIXED)
        s.set_gram_kernel(v)
        s.set_state(X, S, W)
        s.step(prob.K)
        Xg, Sg, Wg = s.get_state()
        us.append(Xg @ Sg @ Wg.T)
        s.close()
    e_fma, e_or = rel_l2(us[1], us[0]), rel_l2(us[1], st.u())
    print(f"tensor-core Grams on {case}: against the FMA Grams {e_fma:.2e}, against the oracle {e_or:.2e}")
    assert 0.0 < e_fma < KERNEL_BOUND[case]
    assert e_or < 1e-3
