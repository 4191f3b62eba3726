"""Pins of the oracle's stencils (Sec. 3.3.2) and the upwind reading of F_S."""
import numpy as np
import pytest

from oracle.grid import apply_D, stencil_matrix


@pytest.mark.parametrize("dims", [(5, 1, 4), (3, 4, 6)])
@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("sign", [-1, 1])
def test_apply_matches_entrywise_matrix(dims, d, sign):
    if dims[1] == 1 and d == 1:
        pytest.skip("no y direction in a slab")
    rng = np.random.default_rng(3)
    n = dims[0] * dims[1] * dims[2]
    Y = rng.standard_normal((n, 3))
    D = stencil_matrix(dims, d, sign, 0.37)
    assert np.abs(apply_D(Y, dims, d, sign, 0.37) - D @ Y).max() < 1e-12


def _bump(x):
    return np.exp(-100.0 * (x - 0.5) ** 2)


def _dbump(x):
    return -200.0 * (x - 0.5) * _bump(x)


@pytest.mark.parametrize("sign", [-1, 1])
def test_second_order_convergence(sign):
    errs = []
    for nx in (128, 256, 512):
        dx = 1.0 / nx
        x = (np.arange(nx) + 0.5) * dx
        out = apply_D(_bump(x)[:, None], (nx, 1, 1), 0, sign, dx)[:, 0]
        errs.append(np.abs(out + _dbump(x)).max())      # D approximates -d/dx
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9)


def test_telescoping_to_boundary_flux():
    rng = np.random.default_rng(4)
    nx, dx = 17, 0.2
    u = rng.standard_normal(nx)
    dm = apply_D(u[:, None], (nx, 1, 1), 0, -1, dx)[:, 0]
    dp = apply_D(u[:, None], (nx, 1, 1), 0, +1, dx)[:, 0]
    # flux form F_{i+1/2} = (3 u_i - u_{i-1})/2 with zero ghosts
    assert abs(dm.sum() * dx + (3 * u[-1] - u[-2]) / 2) < 1e-12
    assert abs(dp.sum() * dx - (3 * u[0] - u[1]) / 2) < 1e-12


def test_literal_pairing_is_unstable_upwind_is_not():
    # 1-D advection with speed +1: the paper pairs D^+ with Lambda^+ (downwind).
    nx, dx = 40, 0.1
    Dp = stencil_matrix((nx, 1, 1), 0, +1, dx)
    Dm = stencil_matrix((nx, 1, 1), 0, -1, dx)
    # periodic symbols (interior behaviour): upwind reading has Re <= 0
    th = np.linspace(0, 2 * np.pi, 721)
    sym_up = -(3 - 4 * np.exp(-1j * th) + np.exp(-2j * th)) / 2      # D^- Lambda^+
    sym_lit = (3 - 4 * np.exp(1j * th) + np.exp(2j * th)) / 2        # D^+ Lambda^+
    assert sym_up.real.max() <= 1e-14
    assert sym_lit.real.max() > 1.0
    # and on the bounded grid: the literal pairing amplifies a smooth pulse, upwind does not
    x = (np.arange(nx) + 0.5) * dx
    u0 = np.exp(-50 * (x - 2.0) ** 2)
    for D, grows in ((Dm, False), (Dp, True)):
        u = u0.copy()
        h = 0.3 * dx
        for _ in range(40):
            k1 = D @ u
            k2 = D @ (u + 0.5 * h * k1)
            k3 = D @ (u + 0.5 * h * k2)
            k4 = D @ (u + h * k3)
            u = u + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        assert (np.linalg.norm(u) > 10 * np.linalg.norm(u0)) == grows


def test_rk4_upwind_cfl_limit():
    # |R(z)| <= 1 over the upwind symbol up to nu ~ 0.696; cfl 0.6 is inside
    th = np.linspace(0, 2 * np.pi, 4001)
    sym = -(3 - 4 * np.exp(-1j * th) + np.exp(-2j * th)) / 2

    def amp(nu):
        z = nu * sym
        return np.abs(1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24).max()

    lo, hi = 0.1, 1.5
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if amp(mid) <= 1 + 1e-12:
            lo = mid
        else:
            hi = mid
    assert 0.68 < lo < 0.71
    assert amp(0.6) <= 1.0 + 1e-12
