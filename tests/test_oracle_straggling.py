"""Pins of the straggling ray model (oracle/straggling.py, Sec. 3.2) against what the
mathematics fixes, independent of the scheme's own formulas:

* the continuous problem d psi/dz = d(S* psi)/dE + (1/2) d/dE(T dpsi/dE) - Sigma psi with
  S* = S + T'/2 moves the mean energy at -S and grows the variance at T(mean) (a Fokker-Planck
  equation in energy): with constant S and T a Gaussian stays Gaussian with mean E0 - S z and
  variance s0^2 + T z. E and E^2 lie in the P2 DG space, so the discrete moments obey the same
  equations; Crank-Nicolson integrates those polynomial-in-z moments exactly;
* the Bohr straggling rate of water against the tabulated constant 0.157 MeV^2 cm^2/g x Z/A;
* absorption alone is the Crank-Nicolson amplification factor, and exp(-Sigma z) to O(h^2);
* without straggling the mean energy follows the CSDA range-energy relation and the energy
  lost to slowing down equals the drop of the integrated energy;
* whole beams: without straggling the DG tracer converges to the independent CSDA tracer of
  oracle/raytrace.py; particle and energy balances close to round-off with straggling.
"""
import numpy as np
import pytest

from oracle import physics as PH
from oracle import straggling as ST


def _gauss(E0, s0):
    return lambda E: np.exp(-0.5 * ((E - E0) / s0) ** 2) / (np.sqrt(2.0 * np.pi) * s0)


def _const(v):
    return lambda E: v + 0.0 * E


def test_bohr_coefficient_matches_the_tabulated_constant():
    # Bohr: d sigma^2 / dx = 0.1569 MeV^2 cm^2 / g x rho Z / A (e.g. the standard
    # 4 pi N_A r_e^2 (m_e c^2)^2 = 0.157 MeV^2 cm^2 / mol per unit Z / A)
    assert abs(ST.t_bohr_water() / (0.1569 * 10.0 / 18.015) - 1.0) < 2e-3
    # the low-energy factor of the reading decreases to the Bohr limit at high energy
    T = ST.straggling_water(np.array([10.0, 50.0, 100.0, 250.0, 1000.0]))
    assert np.all(np.diff(T) < 0) and np.all(T > ST.t_bohr_water())
    assert T[-1] / ST.t_bohr_water() - 1.0 < 5e-3


@pytest.mark.parametrize("S0,T0", [(5.0, 0.5), (2.0, 2.0), (8.0, 0.0)])
def test_constant_coefficients_give_the_exact_moments(S0, T0):
    dg = ST.EnergyDG(50.0, 150.0, 128)
    rm = ST.RayMarch(dg, _const(S0), _const(T0))
    E0, s0, z = 110.0, 2.0, 3.0
    c0 = dg.project(_gauss(E0, s0))
    n0 = dg.number(c0)
    m0, v0 = dg.mean_var(c0)
    c, info = rm.march(c0, [(1.0, 1.0, 0.0), (2.0, 1.0, 0.0)])
    m, v = dg.mean_var(c)
    assert abs(dg.number(c) / n0 - 1.0) < 1e-12
    assert abs(m - (m0 - S0 * z)) < 1e-9 * m0
    assert abs(v - (v0 + T0 * z)) < 1e-9 * v0
    # the energy lost to slowing down is S per unit number and length
    dep = sum(i["deposit"] for i in info)
    assert abs(dep - S0 * z * n0) < 1e-10 * S0 * z


def test_linear_straggling_coefficient_needs_the_drift_correction():
    # T(E) = a + b E: the mean still falls at exactly S and the variance grows at T(mean),
    # var(z) = s0^2 + a z + b (E0 z - S z^2 / 2), only with the drift S* = S + b / 2
    a, b, S0 = 0.2, 0.01, 4.0
    dg = ST.EnergyDG(40.0, 160.0, 128)
    rm = ST.RayMarch(dg, _const(S0), lambda E: a + b * E)
    E0, s0, z = 120.0, 2.5, 4.0
    c0 = dg.project(_gauss(E0, s0))
    m0, v0 = dg.mean_var(c0)
    c, _ = rm.march(c0, [(z, 1.0, 0.0)])
    m, v = dg.mean_var(c)
    assert abs(m - (m0 - S0 * z)) < 1e-9 * m0
    assert abs(v - (v0 + a * z + b * (m0 * z - S0 * z * z / 2.0))) < 1e-8 * v0


def test_gaussian_profile_converges_under_refinement():
    S0, T0, E0, s0, z = 5.0, 0.5, 100.0, 2.0, 2.0
    Es = np.linspace(80.0, 100.0, 201)
    var = s0 ** 2 + T0 * z
    exact = np.exp(-0.5 * (Es - (E0 - S0 * z)) ** 2 / var) / np.sqrt(2.0 * np.pi * var)
    errs = []
    for G in (32, 64, 128):
        dg = ST.EnergyDG(50.0, 150.0, G)
        rm = ST.RayMarch(dg, _const(S0), _const(T0))
        c, _ = rm.march(dg.project(_gauss(E0, s0)), [(z, 1.0, 0.0)])
        errs.append(np.sqrt(np.mean((dg.evaluate(c, Es) - exact) ** 2)) / exact.max())
    assert errs[2] < 1e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_absorption_is_the_crank_nicolson_factor():
    sig, z = 0.8, 1.5
    dg = ST.EnergyDG(50.0, 150.0, 32)
    rm = ST.RayMarch(dg, _const(0.0), _const(0.0), sigma_ref=_const(1.0))
    c0 = dg.project(_gauss(100.0, 3.0))
    c, info = rm.march(c0, [(z, 1.0, sig)])
    h, n = info[0]["h"], info[0]["n_steps"]
    ratio = dg.number(c) / dg.number(c0)
    assert abs(ratio - ((1 - h * sig / 2) / (1 + h * sig / 2)) ** n) < 1e-12
    assert abs(ratio - np.exp(-sig * z)) < (sig * h) ** 2 * sig * z


def test_csda_limit_follows_the_range_energy_relation():
    # no straggling, water power law: a narrow beam's mean energy at depth z is the CSDA energy
    # E(z) = ((R(E0) - z) / alpha)^(1/p) up to the spread's second-order bias
    p, alpha = 1.77, 0.0022
    Sw = lambda E: PH.stopping_power_water(E, p, alpha)
    dg = ST.EnergyDG(20.0, 130.0, 128)
    rm = ST.RayMarch(dg, Sw, _const(0.0))
    E0, s0 = 110.0, 1.0
    c0 = dg.project(_gauss(E0, s0))
    e_in = dg.energy_moment(c0, 1)
    segs = [(1.0, 1.0, 0.0)] * 5
    c, info = rm.march(c0, segs)
    z = 5.0
    E_csda = float(PH.energy_from_range_water(PH.range_water(E0, p, alpha) - z, p, alpha))
    m, v = dg.mean_var(c)
    assert abs(m - E_csda) < 2e-3 * E_csda
    # energy balance: the deposit equals the drop of int E psi (no particle left the interval)
    dep = sum(i["deposit"] for i in info)
    assert abs(dg.number(c) / dg.number(c0) - 1.0) < 1e-12
    assert abs((e_in - dg.energy_moment(c, 1)) - dep) < 1e-10 * e_in
    # and each voxel segment deposits more than the previous one (S rises as E falls)
    d = [i["deposit"] for i in info]
    assert all(d[k + 1] > d[k] for k in range(len(d) - 1))


def test_sipg_operator_is_symmetric_positive_semidefinite():
    dg = ST.EnergyDG(0.0, 10.0, 16)
    K = dg.straggling(lambda E: 0.3 + 0.05 * E)
    assert np.allclose(K, K.T, atol=1e-13)
    w = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert w.min() > -1e-10 * w.max()
    # constants are in its kernel (no flux through the ends, no jumps)
    one = dg.project(lambda E: 1.0 + 0.0 * E)
    assert np.abs(K @ one).max() < 1e-12


def _slab_problem(e_max=66.0):
    from oracle import problem as OP
    from paper_2508_04484_gb300 import workloads as WL
    cfg = WL.base_config(nx=16, ny=1, nz=20, dx=0.2, dy=0.0, dz=0.2, N=3, collision=WL.BOLTZMANN,
                         rank_mode=WL.FIXED, rank=4, rank_max=8, e_max=e_max, e_min=30.0, n_steps=8,
                         precision=WL.FP64, t100=2e-2)
    mats, w = WL.homogeneous(cfg)
    return OP.Problem(cfg, mats, w)


def _pencil(**kw):
    from paper_2508_04484_gb300 import workloads as WL
    return WL.pencil_beam(60.0, (1.3, 0.0, 0.0), (0.2, 0.0, 1.0), **kw)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_without_straggling_the_dg_tracer_converges_to_the_csda_tracer():
    # two independent discretisations of the same CSDA ray (closed-form range-energy segments with
    # nested quadrature, against the energy-DG march): their deposits and fluences converge to each
    # other, and the energy carried into the collided flux agrees to round-off level
    from oracle import raytrace as ORT
    prob = _slab_problem()
    beam = _pencil(spot_sigma=0.0)
    ref = ORT.trace(prob, beam)
    coarse = ST.trace_straggling(prob, beam, n_elem=128, h_max=0.01, straggling=False)
    fine = ST.trace_straggling(prob, beam, n_elem=256, h_max=0.005, straggling=False)
    assert _rel(coarse.e_u, ref.e_u) < 2e-2 and _rel(fine.e_u, ref.e_u) < 2e-3
    assert _rel(coarse.psi.sum(0), ref.psi.sum(0)) < 1.5e-2 and _rel(fine.psi.sum(0), ref.psi.sum(0)) < 1e-3
    assert _rel(fine.psi, ref.psi) < 1.5e-2
    for r in (coarse, fine):
        assert abs(r.removed_energy / ref.removed_energy - 1.0) < 1e-7
        assert abs(r.cutoff_energy / ref.cutoff_energy - 1.0) < 1e-7


@pytest.mark.parametrize("e_max", [60.0, 66.0])
@pytest.mark.parametrize("straggling", [False, True])
def test_tracer_balances_are_exact(e_max, straggling):
    # particles: in = exit + removed + below E_min; energy: in = deposit + removed + exit +
    # E_min x (below E_min) + the no-flux ends' term, to round-off
    prob = _slab_problem(e_max)
    r = ST.trace_straggling(prob, _pencil(spot_sigma=0.1), straggling=straggling)
    V = prob.volume
    n_in = 1.0   # unit beam weight
    assert abs(n_in - (r.removed_particles + r.cutoff_particles + r.exit_particles)) < 1e-12
    e_out = r.e_u.sum() * V + r.removed_energy + r.exit_energy + r.cutoff_energy + r.boundary_energy
    assert abs(r.input_energy - e_out) < 1e-12 * r.input_energy
    # the ends' term is a boundary effect of the scheme: small against the beam's energy
    assert abs(r.boundary_energy) < 1e-4 * r.input_energy
    if not straggling:
        assert r.boundary_energy == 0.0


def test_straggling_spreads_the_energy_distribution_of_a_beam():
    # a 100 MeV beam through 5 cm of water: its energy variance grows by about int T dz
    # (Bohr, plus the growth a falling energy gives an existing spread)
    dg = ST.EnergyDG(20.0, 110.0, 128)
    Sw = lambda E: E ** (1.0 - 1.77) / (1.77 * 0.0022)
    plain = ST.RayMarch(dg, Sw, _const(0.0))
    strag = ST.RayMarch(dg, Sw, ST.straggling_water)
    c0 = dg.project(_gauss(100.0, 0.5))
    c_p, _ = plain.march(c0, [(5.0, 1.0, 0.0)])
    c_s, _ = strag.march(c0, [(5.0, 1.0, 0.0)])
    (m_p, v_p), (m_s, v_s) = dg.mean_var(c_p), dg.mean_var(c_s)
    added = v_s - v_p
    bohr = ST.t_bohr_water() * 5.0
    assert abs(m_s - m_p) < 1e-2
    assert 1.0 * bohr < added < 2.5 * bohr


def test_collided_dose_from_the_dg_source_converges_to_the_csda_one():
    # the whole oracle path with the straggling tracer as the source (straggling off): the
    # low-rank collided solve and its dose converge to those driven by the CSDA tracer
    from oracle import dlra as ODL
    from oracle import problem as OP
    from oracle import raytrace as ORT
    prob = _slab_problem()
    beam = _pencil(spot_sigma=0.0)
    d = np.asarray(beam["dir"]) / np.linalg.norm(beam["dir"])
    ref = ORT.trace(prob, beam)
    r_ref = ODL.solve(prob, [(ref.psi, ref.e_u, d)], ODL.RankControl(mode=OP.FIXED, rank=6))
    errs = []
    for G, h in ((128, 0.01), (256, 0.005)):
        r = ST.trace_straggling(prob, beam, n_elem=G, h_max=h, straggling=False)
        out = ODL.solve(prob, [(r.psi, r.e_u, d)], ODL.RankControl(mode=OP.FIXED, rank=6))
        errs.append((_rel(out["dose"], r_ref["dose"]), _rel(out["dose_collided"], r_ref["dose_collided"])))
    assert errs[0][0] < 2e-2 and errs[1][0] < 1e-3
    assert errs[0][1] < 2e-2 and errs[1][1] < 2e-3
