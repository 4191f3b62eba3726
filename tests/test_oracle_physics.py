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
