"""Uncollided transport with energy straggling along one ray (oracle; test infrastructure only).

Sec. 3.2 of the paper writes the uncollided flux along a ray (depth z) as

    d psi/dz + Sigma_t psi = d(S* psi)/dE + (1/2) d/dE (T d psi/dE),   S* = S + (1/2) dT/dE,

with S the stopping power and T the straggling coefficient; psi(E, z = 0) is the projection of
the beam's (Gaussian) energy distribution. The paper discretises energy by discontinuous
Galerkin with 128 equal elements and polynomials up to degree 2, a Lax-Friedrichs flux for the
slowing-down term and SIPG (symmetric interior penalty) for the straggling term, and integrates
the resulting system M_E dpsi/dz + G psi = 0 in depth by Crank-Nicolson with steps of at most
0.01 cm. This module restates that scheme:

* basis: Legendre polynomials P_0, P_1, P_2 of the element coordinate xi in [-1, 1], so the
  mass matrix is diagonal (Delta / (2j + 1));
* slowing down: element integrals of S* psi dv/dE by 6-point Gauss-Legendre, face flux
  Lax-Friedrichs with alpha = |S*| at the face (for S* > 0 this is the upwind value from the
  higher-energy side); no inflow above E_max, outflow below E_min;
* straggling: SIPG with diffusion coefficient kappa = T / 2, penalty 18 kappa_f / Delta
  (above the 1-D coercivity bound p (p + 1) kappa / Delta for p = 2), no diffusive flux through
  the two ends of the energy interval (a reading: the paper does not state them);
* absorption: element integrals of Sigma_t psi v;
* depth: Crank-Nicolson, (M + h/2 G) c_{n+1} = (M - h/2 G) c_n.

Along a ray the material enters as a factor f(z) >= 0 multiplying S and T (S = f S_ref,
T = f T_ref: both scale with the electron density in Bragg-additivity and Bohr's model) and an
absorption coefficient Sigma_t(E, z) = tau(z) sigma_ref(E), piecewise constant over segments.

Straggling coefficient of water (reading of the paper's Williams formula, whose printed form
lacks the leading term of the bracket): T_w(E) = T_Bohr (1 + 4 I / (3 m_e v^2) ln(2 m_e v^2 / I))
with T_Bohr = 4 pi r_e^2 (m_e c^2)^2 N_e and I = 75 eV; v from the relativistic kinetic energy.

Pins (tests/test_oracle_straggling.py): constant S and T give a Gaussian whose mean falls as
E_0 - S z and whose variance grows as sigma_0^2 + T z (closed form of the continuous problem);
particle number is conserved without absorption; absorption alone reproduces the
Crank-Nicolson factor ((1 - h Sigma/2) / (1 + h Sigma/2))^steps exactly and exp(-Sigma z) to
O(h^2); without straggling the mean energy follows the CSDA range-energy relation of the water
power law; the energy lost to slowing down equals the drop of the integrated energy (energy
balance); the error falls at least at second order under refinement; T_Bohr from its
constants. For whole beams (``trace_straggling``): without straggling it converges to the
independent CSDA tracer ``raytrace.trace`` (deposit 2e-3 and energy-summed fluence 1e-3 at 256
elements and h = 0.005 cm, removed and cut-off energy 1e-7 already at the paper's 128 elements
and 0.01 cm); particle and energy balances are exact with straggling; straggling adds about the
Bohr variance int T dz to a beam's energy spread.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import lu_factor, lu_solve

# physical constants (MeV, cm)
ME_C2 = 0.51099895          # electron rest energy
MP_C2 = 938.27208816        # proton rest energy
R_E = 2.8179403262e-13      # classical electron radius
N_A = 6.02214076e23
I_WATER = 75.0e-6           # mean excitation energy of water
NE_WATER = 1.0 * N_A * 10.0 / 18.015   # electrons per cm^3 (density 1, Z/A = 10/18.015)

_GL_X, _GL_W = np.polynomial.legendre.leggauss(6)


def t_bohr_water():
    """Bohr straggling coefficient of water, 4 pi r_e^2 (m_e c^2)^2 N_e, MeV^2/cm."""
    return 4.0 * np.pi * R_E ** 2 * ME_C2 ** 2 * NE_WATER


def straggling_water(E):
    """T_w(E) for water (the reading above), MeV^2/cm."""
    E = np.asarray(E, dtype=np.float64)
    gamma = 1.0 + E / MP_C2
    beta2 = 1.0 - 1.0 / gamma ** 2
    mv2 = ME_C2 * beta2
    corr = 4.0 * I_WATER / (3.0 * mv2) * np.log(np.maximum(2.0 * mv2 / I_WATER, 1.0))
    return t_bohr_water() * (1.0 + corr)


def _legendre(xi):
    """P_0, P_1, P_2 and their xi-derivatives at the points xi (3 x len(xi) each)."""
    xi = np.asarray(xi, dtype=np.float64)
    P = np.stack([np.ones_like(xi), xi, 0.5 * (3.0 * xi ** 2 - 1.0)])
    dP = np.stack([np.zeros_like(xi), np.ones_like(xi), 3.0 * xi])
    return P, dP


class EnergyDG:
    """The energy discretisation: G elements of P2 Legendre polynomials on [e_min, e_max].

    Coefficients are stored as c[e, j] (element e from the bottom, degree j), flattened
    element-major into vectors of length 3 G.
    """

    def __init__(self, e_min, e_max, n_elem=128):
        self.e_min, self.e_max, self.G = float(e_min), float(e_max), int(n_elem)
        self.delta = (self.e_max - self.e_min) / self.G
        self.edges = self.e_min + self.delta * np.arange(self.G + 1)
        self.centres = 0.5 * (self.edges[:-1] + self.edges[1:])
        self.N = 3 * self.G
        # mass matrix (diagonal): int_e P_i P_j dE = Delta / (2 i + 1) delta_ij
        self.mass = np.tile(self.delta / (2.0 * np.arange(3) + 1.0), self.G)
        # all quadrature points (G x 6), their weights and the basis there (3 x 6)
        self.qE = self.centres[:, None] + 0.5 * self.delta * _GL_X[None, :]
        self.qw = 0.5 * self.delta * _GL_W
        self.qP, _ = _legendre(_GL_X)

    def idx(self, e, j):
        return 3 * e + j

    def quad_points(self, e):
        """Energies and weights (dE) of the element quadrature, and the basis there."""
        E = self.centres[e] + 0.5 * self.delta * _GL_X
        w = 0.5 * self.delta * _GL_W
        P, dP = _legendre(_GL_X)
        return E, w, P, dP * (2.0 / self.delta)

    # ---- projections and moments -------------------------------------------------------
    def project(self, f):
        """L2 projection of the function f(E) (vectorised) onto the DG space."""
        c = np.zeros(self.N)
        for e in range(self.G):
            E, w, P, _ = self.quad_points(e)
            fv = f(E)
            for j in range(3):
                c[self.idx(e, j)] = np.sum(w * fv * P[j]) / self.mass[self.idx(e, j)]
        return c

    def evaluate(self, c, E):
        """psi_h(E) at the energies E (inside [e_min, e_max])."""
        E = np.asarray(E, dtype=np.float64)
        e = np.clip(((E - self.e_min) / self.delta).astype(int), 0, self.G - 1)
        xi = (E - self.centres[e]) / (0.5 * self.delta)
        P, _ = _legendre(xi)
        return sum(c[3 * e + j] * P[j] for j in range(3))

    def number(self, c):
        """int psi dE."""
        return float(np.sum(c[0::3]) * self.delta)

    def energy_moment(self, c, power=1):
        """int E^power psi dE for power 0, 1, 2 (exact for the polynomial pieces)."""
        c0, c1, c2 = c[0::3], c[1::3], c[2::3]
        d, Ec = self.delta, self.centres
        if power == 0:
            return float(np.sum(c0) * d)
        if power == 1:
            return float(np.sum(Ec * d * c0 + d * d * c1 / 6.0))
        if power == 2:
            # (Delta/2) [Ec^2 2 c0 + Ec Delta 2 c1 / 3 + Delta^2/4 (2 c0 / 3 + 4 c2 / 15)]
            return float(np.sum(0.5 * d * (2.0 * Ec ** 2 * c0 + Ec * d * 2.0 * c1 / 3.0
                                           + d * d / 4.0 * (2.0 * c0 / 3.0 + 4.0 * c2 / 15.0))))
        raise ValueError(power)

    def mean_var(self, c):
        n = self.energy_moment(c, 0)
        m1 = self.energy_moment(c, 1) / n
        m2 = self.energy_moment(c, 2) / n
        return m1, m2 - m1 * m1

    def values_at_quadrature(self, c):
        """psi at every quadrature point (G x 6)."""
        return c.reshape(self.G, 3) @ self.qP

    def integral_weighted(self, c, g=None, gq=None):
        """int g(E) psi(E) dE by the element quadrature (g vectorised, or its values gq at the
        quadrature points)."""
        if gq is None:
            gq = g(self.qE)
        return float(np.sum(self.values_at_quadrature(c) * gq * self.qw[None, :]))

    def integrate_interval(self, c, Ea, Eb):
        """int_Ea^Eb psi dE (exact: the Legendre pieces are integrated in closed form)."""
        Ea, Eb = max(Ea, self.e_min), min(Eb, self.e_max)
        if not Eb > Ea:
            return 0.0
        # antiderivatives of P_0, P_1, P_2 in xi: xi, xi^2 / 2, (xi^3 - xi) / 2
        def prim(xi):
            return np.stack([xi, 0.5 * xi ** 2, 0.5 * (xi ** 3 - xi)])
        e0 = min(int((Ea - self.e_min) / self.delta), self.G - 1)
        e1 = min(int((Eb - self.e_min) / self.delta), self.G - 1)
        tot = 0.0
        for e in range(e0, e1 + 1):
            lo = max(Ea, self.edges[e])
            hi = min(Eb, self.edges[e + 1])
            if not hi > lo:
                continue
            xa = (lo - self.centres[e]) / (0.5 * self.delta)
            xb = (hi - self.centres[e]) / (0.5 * self.delta)
            pr = prim(np.array([xb]))[:, 0] - prim(np.array([xa]))[:, 0]
            tot += 0.5 * self.delta * float(c[3 * e:3 * e + 3] @ pr)
        return tot

    def bottom_value(self, c):
        """psi(E_min^+), the trace of the lowest element."""
        return float(c[0] - c[1] + c[2])

    def top_value(self, c):
        """psi(E_max^-), the trace of the highest element."""
        return float(c[-3] + c[-2] + c[-1])

    def project_delta(self, E0):
        """L2 projection of delta(E - E0)."""
        c = np.zeros(self.N)
        e = min(max(int((E0 - self.e_min) / self.delta), 0), self.G - 1)
        xi = (E0 - self.centres[e]) / (0.5 * self.delta)
        P, _ = _legendre(np.array([xi]))
        for j in range(3):
            c[self.idx(e, j)] = P[j, 0] / self.mass[self.idx(e, j)]
        return c

    # ---- operators -----------------------------------------------------------------------
    def _face_values(self, side):
        """Values and derivatives (d/dE) of P_j at the element's bottom (side 0) or top (1)."""
        xi = -1.0 if side == 0 else 1.0
        P, dP = _legendre(np.array([xi]))
        return P[:, 0], dP[:, 0] * (2.0 / self.delta)

    def slowing_down(self, S):
        """Matrix B with (B c)_i = int dE (d/dE (S* psi)) v_i in the DG weak form with the
        Lax-Friedrichs face flux, for the (vectorised) positive function S*(E)."""
        B = np.zeros((self.N, self.N))
        vb, _ = self._face_values(0)
        vt, _ = self._face_values(1)
        for e in range(self.G):
            E, w, P, dP = self.quad_points(e)
            s = S(E)
            # - int S* psi dv/dE
            for i in range(3):
                for j in range(3):
                    B[self.idx(e, i), self.idx(e, j)] -= np.sum(w * s * P[j] * dP[i])
        # faces: F_hat(E_f) [v(E_f^-) from the lower element] - F_hat [v(E_f^+) from the upper]
        for f in range(self.G + 1):
            Ef = self.edges[f]
            sf = float(S(np.array([Ef]))[0])
            alpha = abs(sf)
            lo, hi = f - 1, f        # element below and above the face
            # F_hat = 1/2 s (psi_lo + psi_hi) + 1/2 alpha (psi_hi - psi_lo)
            coef_lo = 0.5 * sf - 0.5 * alpha
            coef_hi = 0.5 * sf + 0.5 * alpha
            for i in range(3):
                # test functions: + F_hat v_lo(top) on the lower element, - F_hat v_hi(bottom)
                rows = []
                if lo >= 0:
                    rows.append((self.idx(lo, i), vt[i]))
                if hi < self.G:
                    rows.append((self.idx(hi, i), -vb[i]))
                for r, sv in rows:
                    for j in range(3):
                        if lo >= 0:
                            B[r, self.idx(lo, j)] += sv * coef_lo * vt[j]
                        if hi < self.G:
                            B[r, self.idx(hi, j)] += sv * coef_hi * vb[j]
        return B

    def straggling(self, T, penalty=18.0):
        """Matrix K with (K c)_i = a_SIPG(psi, v_i) for the diffusion coefficient kappa = T/2
        (so that (1/2) d/dE (T dpsi/dE) contributes -K c); no flux through the ends."""
        K = np.zeros((self.N, self.N))
        for e in range(self.G):
            E, w, P, dP = self.quad_points(e)
            kap = 0.5 * T(E)
            for i in range(3):
                for j in range(3):
                    K[self.idx(e, i), self.idx(e, j)] += np.sum(w * kap * dP[i] * dP[j])
        vb, dvb = self._face_values(0)
        vt, dvt = self._face_values(1)
        for f in range(1, self.G):
            Ef = self.edges[f]
            kf = 0.5 * float(T(np.array([Ef]))[0])
            lo, hi = f - 1, f
            # traces: minus side = lower element's top, plus side = upper element's bottom;
            # jump [u] = u^- - u^+, average {u'} = (u'^- + u'^+) / 2
            val = {lo: vt, hi: -vb}          # contribution of each side to the jump
            der = {lo: 0.5 * dvt, hi: 0.5 * dvb}   # contribution to the average derivative
            sig = penalty * kf / self.delta
            for a in (lo, hi):
                for b in (lo, hi):
                    for i in range(3):
                        for j in range(3):
                            r, c = self.idx(a, i), self.idx(b, j)
                            # - {kappa psi'} [v] - {kappa v'} [psi] + sigma [psi][v]
                            K[r, c] += (-kf * der[b][j] * val[a][i] - kf * der[a][i] * val[b][j]
                                        + sig * val[b][j] * val[a][i])
        return K

    def absorption(self, sigma):
        """Matrix R with (R c)_i = int sigma(E) psi v_i dE."""
        R = np.zeros((self.N, self.N))
        for e in range(self.G):
            E, w, P, _ = self.quad_points(e)
            s = sigma(E)
            for i in range(3):
                for j in range(3):
                    R[self.idx(e, i), self.idx(e, j)] += np.sum(w * s * P[i] * P[j])
        return R


class RayMarch:
    """Crank-Nicolson march of the uncollided energy distribution along a ray.

    S_ref, T_ref: reference stopping power and straggling coefficient (functions of E); a
    segment of material factor f has S = f S_ref, T = f T_ref. sigma_ref: reference removal
    cross section (function of E, or None); a segment's Sigma_t = tau sigma_ref.
    """

    def __init__(self, dg: EnergyDG, S_ref, T_ref, sigma_ref=None, h_max=0.01):
        self.dg = dg
        self.h_max = float(h_max)
        self.S_ref = S_ref
        self.T_ref = T_ref
        # S* = S + (1/2) dT/dE: d/dE of T_ref by central differences of the function
        def s_star(E, eps=1e-4):
            return S_ref(E) + 0.5 * (T_ref(E + eps) - T_ref(E - eps)) / (2.0 * eps)
        self.s_star = s_star
        self.B = dg.slowing_down(s_star)
        self.K = dg.straggling(T_ref)
        self.R = dg.absorption(sigma_ref) if sigma_ref is not None else np.zeros((dg.N, dg.N))
        self.sig_ref_q = sigma_ref(dg.qE) if sigma_ref is not None else np.zeros_like(dg.qE)
        self.M = np.diag(dg.mass)

    def operator(self, f, tau):
        """G with M dc/dz = -G c for material factor f and removal factor tau."""
        return -f * self.B + f * self.K + tau * self.R

    def march(self, c0, segments):
        """Advance c0 through the segments, each (length, f, tau) with Sigma_t = tau sigma_ref,
        or a dict(length, f, R, sig_q) with its own removal matrix R and Sigma_t at the
        quadrature points sig_q (G x 6). Returns the final coefficients and, per segment, a
        dict of integrals over the segment, trapezoidal in z as Crank-Nicolson implies:
        deposit = int int S psi dE dz (energy lost to slowing down), removed_particles and
        removed_energy = int int Sigma_t (1, E) psi dE dz, cutoff_particles = int S*(E_min)
        psi(E_min) dz (outflow below E_min), boundary_energy = int kappa(E_max) psi(E_max) -
        kappa(E_min) psi(E_min) dz (the energy the no-flux ends of the straggling term remove;
        zero without straggling and negligible away from both ends), track = int psi dz
        (coefficients), and n_steps, h, number_in, number_out. With them the balances are exact:
        number_in = number_out + removed_particles + cutoff_particles and int E psi falls by
        deposit + removed_energy + E_min cutoff_particles + boundary_energy."""
        dg = self.dg
        c = np.array(c0, dtype=np.float64)
        out = []
        Sq = self.S_ref(dg.qE)
        # outflow below E_min is S* psi; the no-flux ends of the SIPG form remove energy at the
        # rate kappa (psi(E_max) - psi(E_min)) (kappa = T / 2): tallied so the balance is exact
        Ss_bot = float(self.s_star(np.array([dg.e_min]))[0])
        k_bot = 0.5 * float(self.T_ref(np.array([dg.e_min]))[0])
        k_top = 0.5 * float(self.T_ref(np.array([dg.e_max]))[0])
        for seg in segments:
            if isinstance(seg, dict):
                length, f, R, sig_q = seg["length"], seg["f"], seg["R"], seg["sig_q"]
            else:
                length, f, tau = seg
                R = tau * self.R
                sig_q = tau * self.sig_ref_q if tau != 0.0 else None
            n = max(1, int(np.ceil(length / self.h_max - 1e-12)))
            h = length / n
            G = -f * self.B + f * self.K + (R if R is not None else 0.0)
            A = self.M + 0.5 * h * G
            Bm = self.M - 0.5 * h * G
            lu = lu_factor(A)

            def rates(cc):
                q = dg.values_at_quadrature(cc) * dg.qw[None, :]
                dep = f * float(np.sum(q * Sq))
                if sig_q is None:
                    rp = re = 0.0
                else:
                    rp = float(np.sum(q * sig_q))
                    re = float(np.sum(q * sig_q * dg.qE))
                pb, pt = dg.bottom_value(cc), dg.top_value(cc)
                cut = f * Ss_bot * pb
                bnd = f * (k_top * pt - k_bot * pb)
                return np.array([dep, rp, re, cut, bnd])

            acc = np.zeros(5)
            track = np.zeros_like(c)
            n_in = dg.number(c)
            prev = rates(c)
            for _ in range(n):
                cn = lu_solve(lu, Bm @ c)
                cur = rates(cn)
                acc += 0.5 * h * (prev + cur)
                track += 0.5 * h * (c + cn)
                c, prev = cn, cur
            out.append(dict(n_steps=n, h=h, deposit=acc[0], removed_particles=acc[1], removed_energy=acc[2],
                            cutoff_particles=acc[3], boundary_energy=acc[4], number_in=n_in,
                            number_out=dg.number(c), track=track))
        return c, out


def trace_straggling(prob, beam, n_elem=128, h_max=0.01, straggling=True):
    """The uncollided flux of one beam with energy straggling (Sec. 3.2): the rays of
    ``raytrace.beam_rays`` (transverse positions; the energy spread is carried by the initial
    energy distribution instead of Gauss-Hermite nodes), each marched through its voxel
    segments by ``RayMarch`` with S(x, E) = f(x) S_w(E), T(x, E) = f(x) T_w(E) and
    Sigma_t(x, E) = sum_i w_i(x) Sigma_{t,i}(E) (Eq. mixXS). Returns a ``RayTraceResult`` with
    the same fluence and deposit definitions as ``raytrace.trace`` (bin-averaged fluence per
    energy bin of the collided grid and voxel; energy lost to slowing down per volume), plus
    cutoff_particles, exit_particles and boundary_energy (see ``RayMarch.march``).
    straggling=False sets T = 0 (the CSDA limit)."""
    from . import physics
    from . import raytrace as RT

    p, alpha = prob.phys.p, prob.phys.alpha
    dg = EnergyDG(prob.e_min, prob.e_max, n_elem)
    Sw = lambda E: physics.stopping_power_water(E, p, alpha)
    Tw = straggling_water if straggling else (lambda E: 0.0 * np.asarray(E, dtype=np.float64))
    rm = RayMarch(dg, Sw, Tw, None, h_max)
    Ri = [dg.absorption(lambda E, i=i: prob.phys.sigma_t(i, E)) for i in range(prob.M)]
    sq = [prob.phys.sigma_t(i, dg.qE) for i in range(prob.M)]
    w = np.asarray(prob.w, dtype=np.float64)
    f_cell = np.zeros(prob.n)
    for i, m in enumerate(prob.phys.mats):
        f_cell += w[i] * m.density * m.sp_ratio
    res = RT.RayTraceResult(prob.K, prob.n)
    res.cutoff_particles = 0.0
    res.exit_particles = 0.0
    res.boundary_energy = 0.0
    V = prob.volume
    es = float(beam.get("energy_sigma", 0.0))
    E0 = float(beam["energy"])
    if E0 > prob.e_max + 1e-12:
        raise ValueError("beam energy above e_max")
    if es > 0:
        c0 = dg.project(lambda E: np.exp(-0.5 * ((E - E0) / es) ** 2) / (np.sqrt(2.0 * np.pi) * es))
        c0 /= dg.number(c0)
    else:
        c0 = dg.project_delta(E0)
    flat = dict(beam, energy_sigma=0.0)
    for (o, v, _, wr) in RT.beam_rays(flat, prob):
        segs = RT._segments(o, v, prob)
        if not segs:
            continue
        res.input_energy += wr * dg.energy_moment(c0, 1)
        march = []
        for cell, ta, tb in segs:
            R = sum(w[i, cell] * Ri[i] for i in range(prob.M))
            sig_q = sum(w[i, cell] * sq[i] for i in range(prob.M))
            march.append(dict(length=tb - ta, f=f_cell[cell], R=R, sig_q=sig_q))
        c, info = rm.march(c0, march)
        for (cell, _, _), inf in zip(segs, info):
            res.e_u[cell] += wr * inf["deposit"] / V
            for k in range(prob.K):
                res.psi[k, cell] += wr * dg.integrate_interval(inf["track"], prob.E[k + 1], prob.E[k]) / (V * prob.h)
            res.removed_energy += wr * inf["removed_energy"]
            res.removed_particles += wr * inf["removed_particles"]
            res.cutoff_particles += wr * inf["cutoff_particles"]
            res.cutoff_energy += wr * inf["cutoff_particles"] * prob.e_min
            res.boundary_energy += wr * inf["boundary_energy"]
        res.exit_energy += wr * dg.energy_moment(c, 1)
        res.exit_particles += wr * dg.number(c)
    return res
