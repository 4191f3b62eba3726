"""Uncollided CSDA ray tracer (oracle; test infrastructure only).

Sec. 3.2 of the paper: uncollided protons travel on straight rays; along a ray
the uncollided flux obeys dpsi_u/dz + sum_i w_i Gamma_out,i psi_u = d(S psi_u)/dE
(+ straggling, which this build leaves out: the straggling/DG version is a later
item). Without straggling each ray carries a single energy E(s) with
dE/ds = -S(x, E), and its particle weight decays as dN/ds = -Sigma_t(x, E(s)) N
(Boltzmann; Gamma_out = 0 for Fokker-Planck, Sec. 3.1). The fluence the collided
equation needs is summed over the rays of the beam (Sec. 3.2) and averaged over
each voxel and each energy bin [E_{k+1}, E_k].

Beam model (Sec. 4): Gaussian spot of standard deviation sigma in the plane
perpendicular to the beam and Gaussian energy spread. Discretisation (readings):
* transverse offsets on a uniform grid of pitch min(delta)/4 at half-integer
  positions (j + 1/2) pitch, |offset| < 3.5 sigma, weights exp(-o^2 / 2 sigma^2)
  normalised to the beam weight; a 2-D x-z slab uses one transverse direction;
* transverse axes: u1 = (d_z, 0, -d_x) in a 2-D slab, otherwise
  u1 = normalise(e_ref x d) with e_ref = e_y if |d_y| < 0.9 else e_x, u2 = d x u1;
* energy spread: 5-point Gauss-Hermite nodes when energy_sigma > 0.

Per voxel segment the energy follows from the water range, because every base
material has the water energy dependence (S(x,E) = f(x) S_w(E)):
R_w(E(s)) = R_w(E_in) - f (s - s_in). The particle weight and the fluence and
deposit integrals are evaluated by nested Gauss-Legendre quadrature of their
definitions, written in the energy variable (ds = dE / S(x, E)), which stays
smooth up to the end of the range.

Every branch decides on real parts only, so the tracer also runs on complex mixture
weights: the complex-step derivative Im f(w + i h e) / h (Squire and Trapp, 1998) is then
the exact derivative of this tracer, which ``trace_vjp`` uses for the discrete adjoint.

Pins (tests/test_oracle_raytrace.py): homogeneous water, normal incidence: the
closed form N(s) = exp(-int Sigma_t ds) with E(s) = ((R_0 - s)/alpha)^(1/p); the
energy balance E_in N_in = deposit + removed + exit + cut-off energy; the
direct ODE solution of dE/ds = -S, dN/ds = -Sigma_t N in a heterogeneous slab.
"""
from __future__ import annotations

import math

import numpy as np

from . import physics


def transverse_axes(direction, two_d):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    if two_d:
        u1 = np.array([d[2], 0.0, -d[0]])
        return d, u1 / np.linalg.norm(u1), None
    eref = np.array([0.0, 1.0, 0.0]) if abs(d[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    u1 = np.cross(eref, d)
    u1 /= np.linalg.norm(u1)
    u2 = np.cross(d, u1)
    return d, u1, u2


def beam_rays(beam, prob):
    """List of (origin, direction, energy, weight) for one beam."""
    d, u1, u2 = transverse_axes(beam["dir"], prob.two_d)
    pos = np.asarray(beam["pos"], dtype=np.float64)
    sig = float(beam.get("spot_sigma", 0.0))
    if prob.two_d:
        pitch = min(prob.dx, prob.dz) / 4.0
    else:
        pitch = min(prob.dx, prob.dy, prob.dz) / 4.0
    if sig > 0:
        nh = int(math.ceil(3.5 * sig / pitch))
        offs = (np.arange(-nh, nh) + 0.5) * pitch
        g = np.exp(-0.5 * (offs / sig) ** 2)
    else:
        offs = np.array([0.0])
        g = np.array([1.0])
    if prob.two_d:
        pts = [(pos + o * u1, gw) for o, gw in zip(offs, g)]
    else:
        pts = [(pos + o1 * u1 + o2 * u2, g1 * g2) for o1, g1 in zip(offs, g) for o2, g2 in zip(offs, g)]
    wsum = sum(p[1] for p in pts)
    es = float(beam.get("energy_sigma", 0.0))
    if es > 0:
        xh, wh = np.polynomial.hermite.hermgauss(5)
        enodes = [(beam["energy"] + math.sqrt(2.0) * es * x, wv / math.sqrt(math.pi)) for x, wv in zip(xh, wh)]
    else:
        enodes = [(float(beam["energy"]), 1.0)]
    W = float(beam.get("weight", 1.0))
    rays = []
    for p, gw in pts:
        for e, we in enodes:
            rays.append((p, d, e, W * gw / wsum * we))
    return rays


def _segments(o, v, prob):
    """Voxel segments (cell index, t_a, t_b) of the ray o + t v through the box."""
    L = (prob.nx * prob.dx, prob.ny * prob.dy, prob.nz * prob.dz)
    axes = [0, 2] if prob.two_d else [0, 1, 2]
    t0, t1 = 0.0, np.inf
    for a in axes:
        if abs(v[a]) < 1e-300:
            if o[a] < 0.0 or o[a] > L[a]:
                return []
            continue
        ta = (0.0 - o[a]) / v[a]
        tb = (L[a] - o[a]) / v[a]
        t0 = max(t0, min(ta, tb))
        t1 = min(t1, max(ta, tb))
    if not t1 > t0:
        return []
    ts = [t0, t1]
    nd = {0: prob.nx, 1: prob.ny, 2: prob.nz}
    for a in axes:
        if abs(v[a]) < 1e-300:
            continue
        planes = np.arange(nd[a] + 1) * prob.delta[a]
        tp = (planes - o[a]) / v[a]
        ts.extend(tp[(tp > t0) & (tp < t1)].tolist())
    ts = np.unique(np.array(ts))
    segs = []
    for ta, tb in zip(ts[:-1], ts[1:]):
        if tb - ta <= 1e-14:
            continue
        pm = o + 0.5 * (ta + tb) * v
        i = min(max(int(math.floor(pm[0] / prob.dx)), 0), prob.nx - 1)
        k = min(max(int(math.floor(pm[2] / prob.dz)), 0), prob.nz - 1)
        j = 0 if prob.two_d else min(max(int(math.floor(pm[1] / prob.dy)), 0), prob.ny - 1)
        segs.append(((k * prob.ny + j) * prob.nx + i, ta, tb))
    return segs


class RayTraceResult:
    def __init__(self, K, n, dtype=np.float64):
        self.psi = np.zeros((K, n), dtype=dtype)    # bin-averaged uncollided fluence  [1/(cm^2 MeV)]
        self.e_u = np.zeros(n, dtype=dtype)         # uncollided energy deposit        [MeV/cm^3]
        self.removed_energy = 0.0       # energy carried into the collided flux
        self.removed_particles = 0.0
        self.exit_energy = 0.0          # energy of uncollided protons leaving the box
        self.cutoff_energy = 0.0        # energy of uncollided protons reaching E_min
        self.input_energy = 0.0         # energy entering the box


def trace(prob, beam, nq: int = 12) -> RayTraceResult:
    """Trace one beam through the phantom of ``prob`` (see module docstring)."""
    p, alpha = prob.phys.p, prob.phys.alpha
    res = RayTraceResult(prob.K, prob.n, np.result_type(prob.w, np.float64))
    # material factors per cell
    f_cell = np.zeros(prob.n, dtype=np.result_type(prob.w, np.float64))
    for i, m in enumerate(prob.phys.mats):
        f_cell += prob.w[i] * m.density * m.sp_ratio
    Emin = prob.e_min
    Rmin = physics.range_water(Emin, p, alpha)
    Rbin = physics.range_water(prob.E, p, alpha)   # decreasing with k
    xg, wg = np.polynomial.legendre.leggauss(nq)
    V = prob.volume

    def stopping_cell(cell, E):
        """S(x, E) = sum_i w_i(x) S_i(E) (Eq. mixXS)."""
        out = np.zeros(np.shape(E))
        for i in range(prob.M):
            out = out + prob.w[i, cell] * prob.phys.stopping_power(i, E)
        return out

    def sigma_t_vec(cell, E):
        """Sigma_t(x, E) = sum_i w_i(x) Sigma_{t,i}(E) (Eq. mixXS)."""
        out = np.zeros(np.shape(E))
        for i in range(prob.M):
            out = out + prob.w[i, cell] * prob.phys.sigma_t(i, E)
        return out

    for (o, v, E0, wr) in beam_rays(beam, prob):
        segs = _segments(o, v, prob)
        if not segs:
            continue
        if E0 > prob.e_max + 1e-12:
            raise ValueError("beam energy above e_max")
        R = physics.range_water(E0, p, alpha)
        N = 1.0
        res.input_energy += wr * E0
        alive = True
        for cell, ta, tb in segs:
            f = f_cell[cell]
            ell = tb - ta
            Rb = R - f * ell
            stop = Rb.real <= Rmin
            if stop:
                ell = (R - Rmin) / f
                Rb = Rmin
            # split the segment at bin boundaries (ranges R_k of the grid energies)
            cuts = [0.0]
            inside = Rbin[(Rbin < np.real(R)) & (Rbin > Rb.real)]
            for Rk in sorted(inside, reverse=True):
                cuts.append((R - Rk) / f)
            cuts.append(ell)
            for sa, sb in zip(cuts[:-1], cuts[1:]):
                if np.real(sb - sa) <= 0.0:
                    continue
                Ehi = physics.energy_from_range_water(R - f * sa, p, alpha)
                Elo = physics.energy_from_range_water(R - f * sb, p, alpha)
                kbin = int(np.searchsorted(-prob.E, -0.5 * np.real(Ehi + Elo)) - 1)
                kbin = min(max(kbin, 0), prob.K - 1)
                # integrals over the sub-segment written in the energy variable, ds = dE / S(x, E)
                E = 0.5 * (Ehi - Elo) * xg + 0.5 * (Ehi + Elo)
                wE = 0.5 * (Ehi - Elo) * wg
                Sx = stopping_cell(cell, E)
                NE = np.empty(nq, dtype=res.psi.dtype)
                for j in range(nq):
                    # N(E) = N(Ehi) exp(-int_E^Ehi Sigma_t / S dE')
                    Ei = 0.5 * (Ehi - E[j]) * xg + 0.5 * (Ehi + E[j])
                    wi = 0.5 * (Ehi - E[j]) * wg
                    NE[j] = N * np.exp(-np.sum(wi * sigma_t_vec(cell, Ei) / stopping_cell(cell, Ei)))
                st = sigma_t_vec(cell, E)
                res.psi[kbin, cell] += wr * np.sum(wE * NE / Sx) / (V * prob.h)
                res.e_u[cell] += wr * np.sum(wE * NE) / V
                res.removed_energy += wr * np.sum(wE * st * NE * E / Sx)
                res.removed_particles += wr * np.sum(wE * st * NE / Sx)
                N = N * np.exp(-np.sum(wE * st / Sx))
            R = Rb
            if stop:
                res.cutoff_energy += wr * N * Emin
                alive = False
                break
        if alive:
            res.exit_energy += wr * N * physics.energy_from_range_water(R, p, alpha)
    return res


def crossed_cells(prob, beam):
    """Cells that at least one ray of the beam crosses (the only cells ``trace`` reads)."""
    cells = set()
    for (o, v, _, _) in beam_rays(beam, prob):
        for cell, _, _ in _segments(o, v, prob):
            cells.add(cell)
    return sorted(cells)


def trace_vjp(prob, beam, gpsi, geu, nq: int = 12, h: float = 1e-30):
    """Vector-Jacobian product of ``trace`` with respect to the mixture weights.

    Returns dw (M, n) with dw[i, x] = sum_{k, y} gpsi[k, y] d psi[k, y] / d w_i(x)
    + sum_y geu[y] d e_u[y] / d w_i(x), each derivative taken by the complex step
    Im trace(w + i h e_{i,x}) / h, which has no cancellation, for every cell a ray
    crosses (the tracer reads no other cell, so the derivative is zero there).
    """
    import copy

    dw = np.zeros((prob.M, prob.n))
    pc = copy.copy(prob)
    for i in range(prob.M):
        for x in crossed_cells(prob, beam):
            wc = prob.w.astype(np.complex128)
            wc[i, x] += 1j * h
            pc.w = wc
            r = trace(pc, beam, nq)
            dw[i, x] = (np.sum(gpsi * r.psi.imag) + np.sum(geu * r.e_u.imag)) / h
    return dw
