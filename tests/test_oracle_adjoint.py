"""Pins of the oracle's discrete adjoint (gradients of a loss of the deposited energy).

The paper has no adjoint; the gradient is defined as the derivative of the discrete
forward map (oracle/fullrank.py), so it is pinned against central finite differences of
that map and against the transposes of explicitly assembled operators.
"""
import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import grid as G
from oracle import problem as P
from oracle import raytrace as RT

WATER = dict(density=1.0)
BONE = dict(density=1.85, sp_ratio=0.9, scatter_ratio=1.35, screening=1.5e-3)


def _case(collision="boltzmann", nx=6, ny=1, nz=6, N=3, K=5, seed=1):
    cfg = dict(nx=nx, ny=ny, nz=nz, dx=0.25, dy=0.0 if ny == 1 else 0.25, dz=0.25, N=N, collision=collision,
               e_max=60.0, e_min=40.0, n_steps=K, t100=1e-2)
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.2, 1.0, (2, n))
    w /= w.sum(0)
    mats = [WATER, BONE]
    return cfg, mats, w, (lambda ww: P.Problem(cfg, mats, ww)), rng


@pytest.mark.parametrize("dims", [(5, 1, 4), (3, 4, 5)])
def test_transposed_stencil_is_the_matrix_transpose(dims):
    rng = np.random.default_rng(0)
    n = int(np.prod(dims))
    Y = rng.standard_normal((n, 3))
    for d in (0, 1, 2):
        if dims[1] == 1 and d == 1:
            continue
        for s in (-1, 1):
            D = G.stencil_matrix(dims, d, s, 0.3)
            assert np.abs(D.T @ Y - G.apply_DT(Y, dims, d, s, 0.3)).max() < 1e-12


@pytest.mark.parametrize("ny", [1, 3])
def test_streaming_transpose_identity(ny):
    cfg, mats, w, fac, rng = _case(nx=4, ny=ny, nz=5)
    prob = fac(w)
    y = rng.standard_normal((prob.n, prob.m))
    yb = rng.standard_normal((prob.n, prob.m))
    t = 0.37 * prob.h
    from oracle.fullrank import streaming_rhs
    lhs = np.sum(yb * streaming_rhs(prob, t, y))
    rhs = np.sum(AD.streaming_rhs_T(prob, t, yb) * y)
    assert abs(lhs - rhs) < 1e-12 * np.abs(lhs) + 1e-12


def test_rk4_transpose_identity_and_stopping_derivative():
    cfg, mats, w, fac, rng = _case()
    prob = fac(w)
    from oracle.fullrank import rk4, streaming_rhs
    y0 = rng.standard_normal((prob.n, prob.m))
    yb = rng.standard_normal((prob.n, prob.m))
    ns = 3
    y1 = rk4(lambda t, y: streaming_rhs(prob, t, y), 0.0, y0, prob.h, ns)
    y0b, dw = AD.rk4_vjp(prob, 0.0, y0, prob.h, ns, yb)
    assert abs(np.sum(yb * y1) - np.sum(y0b * y0)) < 1e-11 * abs(np.sum(yb * y1))
    # d<yb, RK4(y0; w)>/dw_i(x) against a central difference in w
    for i, x in [(0, 7), (1, 20)]:
        eps = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i, x] += eps
        wm[i, x] -= eps
        fp = np.sum(yb * rk4(lambda t, y: streaming_rhs(fac(wp), t, y), 0.0, y0, prob.h, ns))
        fm = np.sum(yb * rk4(lambda t, y: streaming_rhs(fac(wm), t, y), 0.0, y0, prob.h, ns))
        fd = (fp - fm) / (2 * eps)
        assert abs(dw[i, x] - fd) < 1e-6 * abs(fd)


def test_raytrace_vjp_matches_finite_differences():
    cfg, mats, w, fac, rng = _case()
    prob = fac(w)
    beam = dict(energy=60.0, pos=[0.7, 0, 0], dir=[0.3, 0, 1], spot_sigma=0.0, weight=1.0)
    r = RT.trace(prob, beam)
    gpsi = rng.standard_normal(r.psi.shape)
    geu = rng.standard_normal(prob.n)
    dw = AD.raytrace.trace_vjp(prob, beam, gpsi, geu)
    cells = RT.crossed_cells(prob, beam)
    assert np.all(dw[:, [c for c in range(prob.n) if c not in cells]] == 0.0)
    for i, x in [(0, cells[0]), (1, cells[3]), (1, cells[-2])]:
        eps = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i, x] += eps
        wm[i, x] -= eps
        rp, rm = RT.trace(fac(wp), beam), RT.trace(fac(wm), beam)
        fd = (np.sum(gpsi * (rp.psi - rm.psi)) + np.sum(geu * (rp.e_u - rm.e_u))) / (2 * eps)
        assert abs(dw[i, x] - fd) < 1e-6 * abs(fd)


@pytest.mark.parametrize("collision", ["boltzmann", "fp"])
def test_gradient_matches_finite_differences_2d(collision):
    cfg, mats, w, fac, rng = _case(collision)
    beams = [dict(energy=60.0, pos=[0.7, 0, 0], dir=[0.3, 0, 1], spot_sigma=0.0, weight=0.8),
             dict(energy=55.0, pos=[1.0, 0, 0], dir=[-0.2, 0, 1], spot_sigma=0.1, weight=1.3)]
    target = rng.uniform(0, 1, w.shape[1])

    def loss(e):
        return 0.5 * np.sum((e - target) ** 2)

    e = AD.loss_and_dose(fac(w), beams)
    g = AD.gradient(fac(w), beams, e - target)
    for i, x in [(0, 8), (1, 8), (0, 14), (1, 20), (1, 2)]:
        fd = AD.finite_difference(fac, beams, w, loss, i, x)
        assert abs(g["dw"][i, x] - fd) < 2e-5 * abs(fd) + 1e-6, (i, x, g["dw"][i, x], fd)
    # the dose is linear in the beam weights: central differences of the quadratic loss are exact
    for b in range(2):
        bp = [dict(bb) for bb in beams]
        bm = [dict(bb) for bb in beams]
        bp[b]["weight"] += 1e-3
        bm[b]["weight"] -= 1e-3
        fd = (loss(AD.loss_and_dose(fac(w), bp)) - loss(AD.loss_and_dose(fac(w), bm))) / 2e-3
        assert abs(g["dbeta"][b] - fd) < 1e-9 * abs(fd)


def test_gradient_matches_finite_differences_3d():
    cfg, mats, w, fac, rng = _case(nx=4, ny=4, nz=5, K=4, seed=3)
    beams = [dict(energy=60.0, pos=[0.55, 0.45, 0], dir=[0.2, 0.1, 1], spot_sigma=0.0, weight=1.0)]
    gx = rng.standard_normal(w.shape[1])

    def loss(e):
        return float(gx @ e)

    g = AD.gradient(fac(w), beams, gx)
    cells = RT.crossed_cells(fac(w), beams[0])
    for i, x in [(0, cells[1]), (1, cells[2]), (0, cells[-1]), (1, 0)]:
        fd = AD.finite_difference(fac, beams, w, loss, i, x)
        assert abs(g["dw"][i, x] - fd) < 2e-5 * abs(fd) + 1e-6, (i, x, g["dw"][i, x], fd)


def test_low_rank_sweep_one_step_is_exact():
    from oracle import dlra as DL
    from oracle import dlra_adjoint as LA
    cfg, mats, w, fac, rng = _case(K=1)
    beams = [dict(energy=60.0, pos=[0.7, 0, 0], dir=[0.3, 0, 1], spot_sigma=0.0, weight=0.8),
             dict(energy=55.0, pos=[1.0, 0, 0], dir=[-0.2, 0, 1], spot_sigma=0.1, weight=1.3)]
    g = rng.standard_normal(w.shape[1])
    ref = AD.gradient(fac(w), beams, g)
    lr = LA.gradient(fac(w), beams, g, DL.RankControl(mode=P.ADAPTIVE, tol=1e-12, r_max=16))
    assert np.linalg.norm(lr["dw"] - ref["dw"]) < 1e-12 * np.linalg.norm(ref["dw"])
    assert np.linalg.norm(lr["dbeta"] - ref["dbeta"]) < 1e-12 * np.linalg.norm(ref["dbeta"])


def test_horner_k_step_equals_classic_rk4():
    from oracle import dlra as DL
    from oracle import dlra_adjoint as LA
    cfg, mats, w, fac, rng = _case(K=3)
    prob = fac(w)
    X, _ = np.linalg.qr(rng.standard_normal((prob.n, 5)))
    W, _ = np.linalg.qr(rng.standard_normal((prob.m, 5)))
    S = np.diag([3.0, 2.0, 1.0, 0.5, 0.2])
    K1 = DL.streaming_bug(prob, X, S, W, 1)[3]
    K1h, v = LA.kstep(prob, X, S, W, 1, False)
    assert np.abs(K1h - K1).max() < 1e-12 * np.abs(K1).max()
    assert len(v) == 4 * prob.n_sub(1)
    # the transposed K-step is the transpose of the forward map: <Y, K(X0)> = <K^T(Y), X0> in the W basis
    Y, _ = np.linalg.qr(rng.standard_normal((prob.n, 5)))
    Kt, _ = LA.kstep(prob, Y, np.eye(5), W, 1, True)
    assert abs(np.sum(Y * K1h) - np.sum(Kt * (X @ S))) < 1e-11 * abs(np.sum(Y * K1h))


def test_low_rank_sweep_converges_to_the_full_rank_gradient():
    from oracle import dlra as DL
    from oracle import dlra_adjoint as LA
    errs = []
    for K in (6, 24):
        cfg, mats, w, fac, rng = _case(nx=8, nz=8, K=K, seed=2)
        x = (np.arange(8) + 0.5) * 0.25
        Xg, Zg = np.meshgrid(x, x)
        g = np.exp(-((Xg - 1.2) ** 2 + (Zg - 1.0) ** 2) / 0.5).ravel()
        beams = [dict(energy=60.0, pos=[1.1, 0, 0], dir=[0.2, 0, 1], spot_sigma=0.1, weight=1.0)]
        ref = AD.gradient(fac(w), beams, g)
        lr = LA.gradient(fac(w), beams, g, DL.RankControl(mode=P.ADAPTIVE, tol=1e-6, r_max=16))
        errs.append(np.linalg.norm(lr["dw"] - ref["dw"]) / np.linalg.norm(ref["dw"]))
    assert errs[1] < 0.2 * errs[0], errs
    assert errs[1] < 1e-2, errs
