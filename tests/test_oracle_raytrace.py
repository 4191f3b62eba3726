"""Pins of the oracle's CSDA ray tracer (Sec. 3.2 without straggling)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

from oracle import physics as ph
from oracle import problem as P
from oracle import raytrace as RT


def _slab_problem(collision, mats, w, nz=30, dz=0.25, K=40, e_max=60.0):
    cfg = dict(nx=4, ny=1, nz=nz, dx=0.5, dy=0.0, dz=dz, N=3, collision=collision,
               e_max=e_max, e_min=1.0, n_steps=K, t100=5e-3)
    return P.Problem(cfg, mats, w)


def test_homogeneous_water_attenuation_closed_form():
    prob = _slab_problem("boltzmann", [dict(density=1.0)], np.ones((1, 4 * 30)), dz=0.2, e_max=100.0)
    beam = dict(energy=100.0, pos=[1.0 + 0.1, 0, 0], dir=[0, 0, 1], spot_sigma=0.0)
    res = RT.trace(prob, beam, nq=16)
    p, alpha = 1.77, 0.0022
    s_unit, xi_unit = ph.screened_rutherford_unit_moments(1e-3, prob.N + 1)
    g0 = s_unit[0] - s_unit[prob.N + 1]
    c = g0 / xi_unit * 0.5 * 5e-3 * 1e4 * p * alpha          # Sigma_t/S_w = c E^(p-3)
    R0 = alpha * 100.0 ** p

    def E_of(s):
        return ((R0 - s) / alpha) ** (1 / p)

    def N_of(s):
        return math.exp(-c * (100.0 ** (p - 2) - E_of(s) ** (p - 2)) / (p - 2))

    L = 30 * 0.2
    assert R0 > L
    assert abs(res.exit_energy / (N_of(L) * E_of(L)) - 1) < 1e-10
    assert abs(res.removed_particles - (1 - N_of(L))) < 1e-10
    # bin-integrated track length of the single ray: sum_x psi V h = int_bin N ds
    Rk = alpha * prob.E ** p
    for k in (0, 5, 17):
        sa, sb = R0 - Rk[k], min(R0 - Rk[k + 1], L)
        if sa >= L:
            continue
        ref = quad(N_of, sa, sb, epsabs=0, epsrel=1e-13)[0]
        got = res.psi[k].sum() * prob.volume * prob.h
        assert abs(got / ref - 1) < 1e-10


@pytest.mark.parametrize("collision", ["boltzmann", "fp"])
def test_energy_balance(collision):
    mats = [dict(density=1.0), dict(density=1.85, sp_ratio=0.9, scatter_ratio=1.35, screening=1.5e-3),
            dict(density=0.26)]
    rng = np.random.default_rng(5)
    w = rng.random((3, 4 * 30))
    w /= w.sum(0, keepdims=True)
    prob = _slab_problem(collision, mats, w)
    beam = dict(energy=45.0, energy_sigma=0.5, pos=[1.0, 0, 0], dir=[0.2, 0, 1], spot_sigma=0.2)
    res = RT.trace(prob, beam)
    tot = res.e_u.sum() * prob.volume + res.removed_energy + res.exit_energy + res.cutoff_energy
    assert abs(tot / res.input_energy - 1) < 1e-12
    if collision == "fp":
        assert res.removed_energy == 0.0
    # every deposited energy goes into bins of the energy grid in order of depth
    assert np.all(res.psi >= 0)


def test_layered_slab_matches_ode():
    # water / bone / lung layers along z; one ray; compare with an ODE solve of
    # dE/ds = -S(x, E), dN/ds = -Sigma_t(x, E) N
    nz, dz = 30, 0.1
    mats = [dict(density=1.0), dict(density=1.85, sp_ratio=0.9, scatter_ratio=1.35, screening=1.5e-3),
            dict(density=0.26)]
    layer = np.repeat([0, 1, 2, 0, 1, 2], 5)
    w = np.zeros((3, nz, 1, 4))
    for k in range(nz):
        w[layer[k], k] = 1.0
    prob = _slab_problem("boltzmann", mats, w.reshape(3, -1), nz=nz, dz=dz, e_max=100.0)
    beam = dict(energy=100.0, pos=[1.1, 0, 0], dir=[0, 0, 1], spot_sigma=0.0)
    res = RT.trace(prob, beam, nq=16)
    p, alpha = 1.77, 0.0022

    def rhs(s, y):
        k = min(int(s / dz), nz - 1)
        i = layer[k]
        E = max(y[0], 1e-6)
        S = prob.phys.stopping_power(i, E)
        st = prob.phys.sigma_t(i, E)
        return [-S, -st * y[1]]

    y = [100.0, 1.0]
    for k in range(nz):
        sol = solve_ivp(rhs, (k * dz, (k + 1) * dz), y, rtol=1e-12, atol=1e-14, method="DOP853")
        y = sol.y[:, -1]
    assert abs(res.exit_energy / (y[0] * y[1]) - 1) < 1e-8


def test_fokker_planck_delta_correction_attenuates_the_beam():
    # with the delta-function corrected Fokker-Planck moments the uncollided beam is removed at
    # Sigma_t = (xi_1/2)(N+1)(N+2) = (T_w/4)(N+1)(N+2): in homogeneous water along a normal ray
    # N(s) = exp(-int Sigma_t ds) in closed form, and the energy balance closes
    cfg = dict(nx=4, ny=1, nz=30, dx=0.5, dy=0.0, dz=0.2, N=3, collision="fp", transport_correction=2,
               e_max=100.0, e_min=1.0, n_steps=40, t100=5e-3)
    prob = P.Problem(cfg, [dict(density=1.0)], np.ones((1, 120)))
    beam = dict(energy=100.0, pos=[1.1, 0, 0], dir=[0, 0, 1], spot_sigma=0.0)
    res = RT.trace(prob, beam, nq=16)
    p, alpha, N = 1.77, 0.0022, 3
    c = 0.25 * (N + 1) * (N + 2) * 5e-3 * 1e4 * p * alpha      # Sigma_t / S_w = c E^(p-3)
    R0 = alpha * 100.0 ** p
    L = 30 * 0.2
    E_L = ((R0 - L) / alpha) ** (1 / p)
    N_L = math.exp(-c * (100.0 ** (p - 2) - E_L ** (p - 2)) / (p - 2))
    assert abs(res.removed_particles - (1 - N_L)) < 1e-10
    tot = res.e_u.sum() * prob.volume + res.removed_energy + res.exit_energy + res.cutoff_energy
    assert abs(tot / res.input_energy - 1) < 1e-12
    assert res.removed_energy > 0.1 * res.input_energy
