"""Pins of the oracle's physics coefficients (Sec. 2.1, Sec. 2.1.1, Sec. 3.3.1)."""
import math

import numpy as np
import pytest

from oracle import physics as ph


@pytest.mark.parametrize("eta", [1e-3, 1.5e-3, 1e-2])
def test_screened_rutherford_closed_forms(eta):
    s, xi = ph.screened_rutherford_unit_moments(eta, 3)
    assert abs(s[0] / (math.pi / (eta * (1 + eta))) - 1) < 1e-12
    assert abs(xi / (2 * math.pi * (math.log((1 + eta) / eta) - 1 / (1 + eta))) - 1) < 1e-12
    # xi_1 = sigma_0 - sigma_1 (P_1(mu) = mu)
    assert abs((s[0] - s[1]) / xi - 1) < 1e-12


@pytest.mark.parametrize("eta", [1e-3, 2e-3])
def test_legendre_q_identity(eta):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    s, _ = ph.screened_rutherford_unit_moments(eta, 22)
    a = mp.mpf(1) + 2 * mp.mpf(eta)
    for l in (0, 1, 2, 7, 15, 16, 21, 22):
        q = mp.diff(lambda z: mp.legenq(l, 0, z, type=3), a)
        ref = float(mp.re(-4 * mp.pi * q))
        assert abs(s[l] / ref - 1) < 1e-12


def test_range_is_integral_of_inverse_stopping_power():
    p, alpha = 1.77, 0.0022
    for E in (5.0, 50.0, 150.0):
        h = 1e-4 * E
        dR = (ph.range_water(E + h, p, alpha) - ph.range_water(E - h, p, alpha)) / (2 * h)
        assert abs(dR * ph.stopping_power_water(E, p, alpha) - 1) < 1e-8
    # Bragg-Kleeman range of 100 MeV protons in water (alpha 100^p)
    assert abs(ph.range_water(100.0, p, alpha) - 0.0022 * 100 ** 1.77) < 1e-12


def test_material_tables_fp_and_boltzmann():
    mats = [ph.Material(1.0), ph.Material(1.85, 0.9, 1.35, 1.5e-3)]
    N = 7
    fp = ph.PhysicsTables(mats, N, ph.FOKKER_PLANCK, 0, 1.77, 0.0022, 1.72e-4)
    bz = ph.PhysicsTables(mats, N, ph.BOLTZMANN, 1, 1.77, 0.0022, 1.72e-4)
    E = 80.0
    l = np.arange(N + 1)
    G, St = fp.moments(1, E)
    assert St == 0.0
    assert np.allclose(G, -0.5 * fp.xi1(1, E) * l * (l + 1))
    # Boltzmann: transport correction shifts G and Sigma_t equally; self-scattering unchanged
    bz0 = ph.PhysicsTables(mats, N, ph.BOLTZMANN, 0, 1.77, 0.0022, 1.72e-4)
    assert np.allclose(bz.self_scatter(1, E), bz0.self_scatter(1, E), rtol=1e-13, atol=0)
    sig = bz.boltzmann_moments(1, E)
    assert np.allclose(bz.inscatter(1, E), sig[: N + 1] - sig[N + 1])
    assert abs(bz.sigma_t(1, E) - (sig[0] - sig[N + 1])) < 1e-15 * sig[0]
    # sigma_0 - sigma_1 equals xi_1 of the material
    assert abs((sig[0] - sig[1]) / bz.xi1(1, E) - 1) < 1e-12


def _exponential_kernel_etc_moments(eps, N):
    """Unit-xi_1 moments of the kernel exp(-(1 - mu)/eps) under the extended transport
    correction, by Gauss-Legendre quadrature in x = 1 - mu on graded panels (independent of the
    oracle's kernels): returns (sigma_l - sigma_{N+1}) / xi_1 for l = 0..N."""
    xg, wg = np.polynomial.legendre.leggauss(40)
    edges = [0.0]
    h = eps / 8
    while edges[-1] + h < 2.0:
        edges.append(edges[-1] + h)
        h *= 1.5
    edges.append(2.0)
    mu, w = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        mu.append(1.0 - (0.5 * (b - a) * xg + 0.5 * (b + a)))
        w.append(0.5 * (b - a) * wg)
    mu, w = np.concatenate(mu), np.concatenate(w)
    k = np.exp(-(1.0 - mu) / eps)
    sig = np.array([2 * np.pi * np.sum(w * np.polynomial.legendre.legval(mu, np.eye(N + 2)[l]) * k)
                    for l in range(N + 2)])
    xi = 2 * np.pi * np.sum(w * (1.0 - mu) * k)
    return (sig[: N + 1] - sig[N + 1]) / xi


def test_delta_corrected_fokker_planck_is_the_forward_peaked_limit():
    # the corrected Fokker-Planck moments (xi/2)[(N+1)(N+2) - l(l+1)] are what the extended
    # transport correction gives for a Boltzmann kernel in the forward-peaked limit at fixed xi_1:
    # the difference falls linearly with the kernel width
    N = 5
    l = np.arange(N + 1)
    limit = 0.5 * ((N + 1) * (N + 2) - l * (l + 1))
    errs = [np.abs(_exponential_kernel_etc_moments(eps, N) - limit).max() / limit.max()
            for eps in (1e-2, 1e-3, 1e-4)]
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 8 and errs[2] < 1e-3
    # the oracle's tables with the correction flag (2)
    mats = [ph.Material(1.0), ph.Material(1.85, 0.9, 1.35, 1.5e-3)]
    fp = ph.PhysicsTables(mats, N, ph.FOKKER_PLANCK, 2, 1.77, 0.0022, 1.72e-4)
    fp0 = ph.PhysicsTables(mats, N, ph.FOKKER_PLANCK, 0, 1.77, 0.0022, 1.72e-4)
    E = 70.0
    xi = fp.xi1(1, E)
    G, St = fp.moments(1, E)
    assert np.abs(G / xi - _exponential_kernel_etc_moments(1e-5, N)).max() < 1e-4 * limit.max()
    assert St == G[0] and abs(fp.sigma_t(1, E) - G[0]) < 1e-15 * G[0]
    # the degree N+1 moment of the corrected expansion vanishes; self-scattering is unchanged
    assert abs(0.5 * xi * ((N + 1) * (N + 2) - (N + 1) * (N + 2))) == 0.0
    assert np.allclose(fp.self_scatter(1, E), fp0.self_scatter(1, E), rtol=1e-13, atol=0)
    # the value 1 keeps the uncorrected Fokker-Planck moments (the extended transport correction
    # applies to the Boltzmann moments only)
    fp1 = ph.PhysicsTables(mats, N, ph.FOKKER_PLANCK, 1, 1.77, 0.0022, 1.72e-4)
    assert np.array_equal(fp1.moments(1, E)[0], fp0.moments(1, E)[0]) and fp1.sigma_t(1, E) == 0.0
