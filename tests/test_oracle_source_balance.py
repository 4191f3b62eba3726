"""Pins of the oracle's first-collision source beyond its l = 0 entry, and of the collided
energy balance (Sec. 3.3.1 Eq. discAngle, Sec. 3.3.3 steps 2-4; Sec. 2.1 CSDA energy loss).

The source of a beam with direction Omega_in is Q = A B^T with B[p, i] = G_{i,l(p)} m_p(Omega_in).
Its angular factor is checked against quantities that do not go through the oracle's formula:

* the real harmonics of degree <= 2 written as Cartesian polynomials of Omega (textbook forms);
* Boltzmann: the moments of the in-scattered distribution Sigma_s(Omega . Omega_in), integrated
  over the sphere by a product rule in a frame about Omega_in (no Legendre expansion), with the
  kernel amplitude from the closed form of xi_1 for the screened Rutherford kernel;
* Fokker-Planck: (xi_1 / 2) times the Laplace-Beltrami operator of each harmonic at Omega_in,
  by central differences in spherical coordinates;
* the collided current sum_x (u_x, u_y, u_z) points downstream along an oblique 3-D beam.

Planted mistakes (a sign flip of the k < 0 harmonics at Omega_in, m(-Omega_in), G_0 used for
every degree) each fail at least one of these pins.

Energy balance: with N_k = sum_x V sqrt(4 pi) u_0(x) the collided particles, Src_k the particles
the source adds in step k and O_k the particles streaming removes through the boundary in step k,
the deposit accumulated after every step satisfies exactly sum_x V e_c = sum_k (Src_k - O_k)
(E_k - E_K); the source hands over the tracer's removed particles and energy to O(dE^2); the whole
energy of the beam E_0 = deposits + uncollided exit and cut-off + energy streamed out + E_min N_K
holds up to the first-order splitting bias dE/2 per collided particle.
"""
import math

import numpy as np
import pytest

from oracle import angular as AN
from oracle import dlra as DL
from oracle import fullrank as FR
from oracle import problem as P
from oracle import raytrace as RT

SQ4PI = math.sqrt(4.0 * math.pi)
_C0 = 1.0 / SQ4PI
_C1 = math.sqrt(3.0 / (4.0 * math.pi))
_C2 = math.sqrt(15.0 / (4.0 * math.pi))
_C20 = math.sqrt(5.0 / (16.0 * math.pi))
_C22 = math.sqrt(15.0 / (16.0 * math.pi))


def cartesian_harmonics(o):
    """Real harmonics of degree 0..2 at the unit vector o, ordered p = l^2 + l + k."""
    x, y, z = o
    return np.array([_C0, _C1 * y, _C1 * z, _C1 * x, _C2 * x * y, _C2 * y * z, _C20 * (3 * z * z - 1),
                     _C2 * x * z, _C22 * (x * x - y * y)])


OMEGA_IN = np.array([0.5, -0.4, 0.77]) / np.linalg.norm([0.5, -0.4, 0.77])
DENSITY, KAPPA, ETA, T100 = 1.3, 1.2, 0.2, 2e-2


def _problem(collision, **kw):
    cfg = dict(nx=4, ny=3, nz=5, dx=0.25, dy=0.25, dz=0.25, N=4, collision=collision, e_max=60.0, e_min=50.0,
               n_steps=4, t100=T100, transport_correction=0)
    cfg.update(kw)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    mat = dict(density=DENSITY, scatter_ratio=KAPPA, screening=ETA)
    return P.Problem(cfg, [mat], np.ones((1, n)))


def _xi1(E):
    return DENSITY * KAPPA * 0.5 * T100 * (100.0 / E) ** 2


def boltzmann_source_error():
    """Relative max difference of B[:9] from the sphere integral of the screened kernel."""
    prob = _problem("boltzmann")
    k = 1
    _, B = FR.source_factors(prob, k, np.ones(prob.n), OMEGA_IN)
    E = 0.5 * (prob.E[k] + prob.E[k + 1])
    # kernel C / (1 - mu + 2 eta)^2 with C from xi_1 = 2 pi C [ln((1 + eta)/eta) - 1/(1 + eta)]
    C = _xi1(E) / (2.0 * math.pi * (math.log((1.0 + ETA) / ETA) - 1.0 / (1.0 + ETA)))
    e1 = np.cross([0.0, 1.0, 0.0], OMEGA_IN)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(OMEGA_IN, e1)
    xs, ws = np.polynomial.legendre.leggauss(200)
    nphi = 16
    q = np.zeros(9)
    for mu, wm in zip(xs, ws):
        s = math.sqrt(1.0 - mu * mu)
        kern = C / (1.0 - mu + 2.0 * ETA) ** 2
        for j in range(nphi):
            ph = (j + 0.5) * 2.0 * math.pi / nphi
            o = mu * OMEGA_IN + s * (math.cos(ph) * e1 + math.sin(ph) * e2)
            q += wm * (2.0 * math.pi / nphi) * kern * cartesian_harmonics(o)
    return float(np.abs(B[:9, 0] - q).max() / np.abs(q).max())


def fokker_planck_source_error():
    """Relative max difference of B[:9] from (xi_1/2) (Laplace-Beltrami of m_p)(Omega_in)."""
    prob = _problem("fp")
    k = 1
    _, B = FR.source_factors(prob, k, np.ones(prob.n), OMEGA_IN)
    E = 0.5 * (prob.E[k] + prob.E[k + 1])

    def f(th, ph):
        return cartesian_harmonics([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])

    th0 = math.acos(OMEGA_IN[2])
    ph0 = math.atan2(OMEGA_IN[1], OMEGA_IN[0])
    h = 1e-4
    d_th = (math.sin(th0 + h / 2) * (f(th0 + h, ph0) - f(th0, ph0))
            - math.sin(th0 - h / 2) * (f(th0, ph0) - f(th0 - h, ph0))) / (h * h * math.sin(th0))
    d_ph = (f(th0, ph0 + h) - 2.0 * f(th0, ph0) + f(th0, ph0 - h)) / (h * h * math.sin(th0) ** 2)
    expect = 0.5 * _xi1(E) * (d_th + d_ph)
    return float(np.abs(B[:9, 0] - expect).max() / np.abs(expect).max())


def collided_current_cosine():
    """Cosine between the total collided current after 3 energy steps and Omega_in (3-D,
    full rank, Boltzmann with the transport correction)."""
    cfg = dict(nx=6, ny=6, nz=6, dx=0.25, dy=0.25, dz=0.25, N=3, collision="boltzmann", e_max=60.0, e_min=54.0,
               n_steps=3, t100=T100)
    prob = P.Problem(cfg, [dict(density=1.0)], np.ones((1, 216)))
    beam = dict(energy=60.0, pos=[0.6, 0.9, 0.0], dir=list(OMEGA_IN), spot_sigma=0.15)
    r = RT.trace(prob, beam)
    u = FR.solve(prob, [(r.psi, r.e_u, OMEGA_IN)])["u"]
    # m_1 = sqrt(3/4pi) (Omega_y, Omega_z, Omega_x) at p = 1, 2, 3
    J = np.array([u[:, 3].sum(), u[:, 1].sum(), u[:, 2].sum()])
    return float(J @ OMEGA_IN / np.linalg.norm(J))


def test_real_harmonics_match_cartesian_forms():
    rng = np.random.default_rng(1)
    for _ in range(20):
        o = rng.standard_normal(3)
        o /= np.linalg.norm(o)
        assert np.abs(AN.real_sh_dir(2, o) - cartesian_harmonics(o)).max() < 1e-14


def test_streaming_matrices_couple_l0_to_the_matching_l1_harmonic():
    # A_d[0, p] = int m_0 m_p Omega_d = 1/sqrt(3) for the harmonic proportional to Omega_d
    # (p = 3 for x, 1 for y, 2 for z) and 0 otherwise: the basis of A_d and of m(Omega_in) agree
    A = AN.streaming_matrices(3)
    for d, p in ((0, 3), (1, 1), (2, 2)):
        row = A[d][0].copy()
        assert abs(row[p] - 1.0 / math.sqrt(3.0)) < 1e-14
        row[p] = 0.0
        assert np.abs(row).max() < 1e-14


def test_boltzmann_source_moments_equal_the_sphere_integral():
    assert boltzmann_source_error() < 1e-10


def test_fokker_planck_source_moments_equal_the_laplace_beltrami():
    assert fokker_planck_source_error() < 1e-6


def test_collided_current_points_downstream():
    assert collided_current_cosine() > 0.9


def _flip_negative_orders(N, omega):
    m = _real_sh_dir(N, omega)
    for l in range(N + 1):
        for k in range(-l, 0):
            m[AN.moment_index(l, k)] *= -1.0
    return m


_real_sh_dir = AN.real_sh_dir
_inscatter = P.Problem.inscatter_coefficients


def _g0_everywhere(self, k):
    g = _inscatter(self, k)
    return np.repeat(g[:, :1], g.shape[1], axis=1)


PLANTS = {
    "k<0 sign flipped at Omega_in": lambda mp: mp.setattr(AN, "real_sh_dir", _flip_negative_orders),
    "m(-Omega_in)": lambda mp: mp.setattr(AN, "real_sh_dir", lambda N, o: _real_sh_dir(N, -np.asarray(o))),
    "G_0 for every degree": lambda mp: mp.setattr(P.Problem, "inscatter_coefficients", _g0_everywhere),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_source_mistake_fails_a_pin(plant, monkeypatch):
    PLANTS[plant](monkeypatch)
    failed = [boltzmann_source_error() > 1e-10, fokker_planck_source_error() > 1e-6]
    if plant == "m(-Omega_in)":
        failed.append(collided_current_cosine() <= 0.9)
        assert all(failed)
    assert any(failed)


# ---------------------------------------------------------------------------------------------
# energy balance
# ---------------------------------------------------------------------------------------------

def _slab(collision, K):
    cfg = dict(nx=16, ny=1, nz=16, dx=0.25, dy=0.0, dz=0.25, N=3, collision=collision, e_max=60.0, e_min=1.0,
               n_steps=K, t100=T100)
    prob = P.Problem(cfg, [dict(density=1.0)], np.ones((1, 256)))
    beam = dict(energy=58.0, pos=[1.9, 0.0, 0.0], dir=[0.15, 0.0, 1.0], spot_sigma=0.3)
    r = RT.trace(prob, beam)
    d = np.asarray(beam["dir"]) / np.linalg.norm(beam["dir"])
    return prob, r, [(r.psi, r.e_u, d)]


def _budget_full_rank(prob, r, src):
    """Per step: particles before, removed by streaming (boundary), added by the source; and
    the collided deposit, from the oracle's own building blocks in the order of its solve."""
    V = prob.volume
    u = np.zeros((prob.n, prob.m))
    e_c = np.zeros(prob.n)
    out, add = [], []
    for k in range(prob.K):
        n0 = V * SQ4PI * u[:, 0].sum()
        us = FR.rk4(lambda t, y: FR.streaming_rhs(prob, t, y), k * prob.h, u, prob.h, prob.n_sub(k))
        out.append(n0 - V * SQ4PI * us[:, 0].sum())
        u = us / (1.0 - FR.scatter_factor(prob, k))
        A, B = FR.source_factors(prob, k, r.psi[k], src[0][2])
        q = prob.h * (A @ B.T)
        add.append(V * SQ4PI * q[:, 0].sum())
        u = u + q
        e_c += prob.h * SQ4PI * u[:, 0]
    return np.array(out), np.array(add), e_c, V * SQ4PI * u[:, 0].sum()


@pytest.mark.parametrize("collision", ["boltzmann", "fp"])
def test_collided_deposit_equals_the_particle_budget(collision):
    # exact discrete identity: every collided particle deposits dE per energy step until E_K
    prob, r, src = _slab(collision, 59)
    out, add, e_c, _ = _budget_full_rank(prob, r, src)
    fr = FR.solve(prob, src)
    assert np.abs(e_c - fr["dose_collided"]).max() <= 1e-14 * np.abs(e_c).max()
    lhs = prob.volume * fr["dose_collided"].sum()
    rhs = np.sum((add - out) * (prob.E[:-1] - prob.E[-1]))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_source_hands_over_the_removed_particles_and_energy():
    # the source of bin k is sigma_0(E_{k+1/2}) times the bin-averaged fluence: a midpoint rule
    # of the tracer's removal, second order in dE
    errs = []
    for K in (59, 118):
        prob, r, src = _slab("boltzmann", K)
        _, add, _, _ = _budget_full_rank(prob, r, src)
        Emid = 0.5 * (prob.E[:-1] + prob.E[1:])
        ep = add.sum() / r.removed_particles - 1.0
        ee = (add * Emid).sum() / r.removed_energy - 1.0
        errs.append((abs(ep), abs(ee)))
    assert errs[0][0] < 2e-3 and errs[0][1] < 5e-4
    assert errs[0][0] / errs[1][0] > 3.0 and errs[0][1] / errs[1][1] > 3.0


@pytest.mark.parametrize("solver", ["full", "dlra"])
def test_global_energy_balance(solver):
    # E_0 = sum V (e_u + e_c) + uncollided exit and cut-off energy + energy streamed out
    # + E_min N_K, up to dE/2 per collided particle (the source enters at the end of its step)
    # and O(dE^2); the low-rank solve holds it to its truncation level
    res = []
    for K in (59, 118):
        prob, r, src = _slab("boltzmann", K)
        V = prob.volume
        Emid = 0.5 * (prob.E[:-1] + prob.E[1:])
        if solver == "full":
            out, add, e_c, n_end = _budget_full_rank(prob, r, src)
        else:
            st = DL.State(prob.n, prob.m)
            rc = DL.RankControl(mode=P.ADAPTIVE, tol=1e-6, r_max=16)
            n0, out, add, e_c = 0.0, [], [], np.zeros(prob.n)
            for k in range(prob.K):
                DL.step(prob, st, k, src, rc)
                A, B = FR.source_factors(prob, k, r.psi[k], src[0][2])
                a = prob.h * V * SQ4PI * (A @ B[0]).sum()
                n1 = V * SQ4PI * st.moment0().sum()
                add.append(a)
                out.append(n0 + a - n1)
                n0 = n1
                e_c += prob.h * SQ4PI * st.moment0()
            out, add, n_end = np.array(out), np.array(add), n0
            ref = FR.solve(prob, src)["dose_collided"]
            assert abs(e_c.sum() / ref.sum() - 1.0) < 1e-2
        total = (V * (e_c.sum() + r.e_u.sum()) + r.exit_energy + r.cutoff_energy + np.sum(out * Emid)
                 + prob.E[-1] * n_end)
        bias = 0.5 * prob.h * add.sum()
        res.append((total - r.input_energy) / r.input_energy)
        assert abs(total - bias - r.input_energy) < 5e-4 * r.input_energy
    # the remaining imbalance is the first-order splitting bias: it halves with dE
    assert 1.7 < res[0] / res[1] < 2.3
