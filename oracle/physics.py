"""Physics coefficients (oracle; test infrastructure only).

Sec. 2.1 / Sec. 2.1.1 of the paper define the CSDA model with stopping power S,
the Boltzmann collision operator with differential cross section Sigma_s, the
Fokker-Planck operator (xi_1 / 2) L with the first transport coefficient
xi_1 = 2 pi int (1 - mu) Sigma_s dmu, and the mixture (Bragg additivity) rule
Sigma(x, E) = sum_i w_i(x) Sigma_i(E) (Eq. mixXS). Sec. 3.3.1 defines the
scattering moments G_{i,pp} = 2 pi int P_l(mu) Sigma_{s;i} dmu (Boltzmann) and
G_{i,pp} = -(xi_{1;i}/2) l (l+1) (Fokker-Planck), with Sigma_t = G_{i,00}.

The paper's own data (TOPAS stopping powers, Moliere cross sections of 12
elements) is not available. The synthetic stand-ins, all stated as inputs:

* water stopping power: Bragg-Kleeman S_w(E) = E^(1-p) / (p alpha), range
  R_w(E) = alpha E^p (the integral of 1/S_w);
* scattering power T_w(E) = t100 (100 MeV / E)^2 rad^2/cm, xi_1 = T / 2;
* base material i: S_i = rho_i s_i S_w(E), xi_{1;i} = rho_i kappa_i T_w(E) / 2;
* Boltzmann kernel of material i: screened Rutherford
  Sigma_{s;i}(E, mu) = C_i(E) / (1 - mu + 2 eta_i)^2, with C_i fixed by xi_{1;i};
* extended transport correction (Sec. 3.3.1, flag): sigma_l <- sigma_l - sigma_{N+1};
* the delta-function corrected expansion of the Fokker-Planck moments (Sec. 3.3.1, the
  correction of Landesman and Morel; flag value 2): the moments are shifted by the same
  constant so that the degree N+1 moment vanishes, G_l = (xi_1/2) [(N+1)(N+2) - l(l+1)],
  with Sigma_t = G_0 = (xi_1/2)(N+1)(N+2); the self-scattering G_l - Sigma_t is unchanged.
  These are the small-screening limit of the screened-Rutherford moments under the extended
  transport correction (pinned in tests/test_oracle_physics.py).

Every moment here is computed by quadrature of its defining integral. Pins
(tests/test_oracle_physics.py): the closed forms sigma_0 = pi C / (eta (1+eta))
and xi_1 = 2 pi C [ln((1+eta)/eta) - 1/(1+eta)], the Legendre-Q identity
sigma_l = -4 pi C Q_l'(1 + 2 eta) evaluated with mpmath, sigma_0 - sigma_1 = xi_1,
and the range/stopping-power identity dR/dE = 1/S.
"""
from __future__ import annotations

import numpy as np

FOKKER_PLANCK = 0
BOLTZMANN = 1


def _num(x):
    """x as a float64 array, or complex128 when x is complex (complex-step derivatives)."""
    x = np.asarray(x)
    return x.astype(np.result_type(x, np.float64))


def stopping_power_water(E, p, alpha):
    """S_w(E) = E^(1-p) / (p alpha)  [MeV/cm]."""
    E = _num(E)
    return E ** (1.0 - p) / (p * alpha)


def range_water(E, p, alpha):
    """CSDA range R_w(E) = int_0^E dE'/S_w(E') = alpha E^p  [cm]."""
    E = _num(E)
    return alpha * E ** p


def energy_from_range_water(R, p, alpha):
    R = _num(R)
    return (np.where(np.real(R) > 0.0, R, 0.0) / alpha) ** (1.0 / p)


def scattering_power_water(E, t100):
    """T_w(E) = t100 (100/E)^2  [rad^2/cm]."""
    E = _num(E)
    return t100 * (100.0 / E) ** 2


def _graded_panels(eta):
    """Panels in x = 1 - mu on [0, 2], geometrically graded toward x = 0."""
    edges = [0.0]
    h = eta / 16.0
    while edges[-1] + h < 2.0:
        edges.append(edges[-1] + h)
        h *= 2.0
    edges.append(2.0)
    return np.array(edges)


def _kernel_quadrature(eta, npts=24):
    """Nodes (mu) and weights for int_{-1}^{1} f(mu) dmu, graded for the screened kernel."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    edges = _graded_panels(eta)
    xs, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (b - a) * xg + 0.5 * (b + a))
        ws.append(0.5 * (b - a) * wg)
    x = np.concatenate(xs)
    return 1.0 - x, np.concatenate(ws)


def screened_rutherford_unit_moments(eta, lmax):
    """For the kernel k(mu) = 1 / (1 - mu + 2 eta)^2 (unit amplitude):
    returns (s_l = 2 pi int P_l k dmu for l = 0..lmax, xi = 2 pi int (1-mu) k dmu),
    both by graded Gauss-Legendre quadrature of the definitions.
    """
    mu, wq = _kernel_quadrature(eta)
    k = 1.0 / (1.0 - mu + 2.0 * eta) ** 2
    out = np.zeros(lmax + 1)
    for l in range(lmax + 1):
        c = np.zeros(l + 1)
        c[l] = 1.0
        out[l] = 2 * np.pi * np.sum(wq * np.polynomial.legendre.legval(mu, c) * k)
    xi = 2 * np.pi * np.sum(wq * (1.0 - mu) * k)
    return out, xi


class Material:
    def __init__(self, density, sp_ratio=1.0, scatter_ratio=1.0, screening=1e-3):
        self.density = float(density)
        self.sp_ratio = float(sp_ratio)
        self.scatter_ratio = float(scatter_ratio)
        self.screening = float(screening)

    @staticmethod
    def from_dict(d):
        return Material(d["density"], d.get("sp_ratio", 1.0), d.get("scatter_ratio", 1.0),
                        d.get("screening", 1e-3))


class PhysicsTables:
    """Per-material coefficients as functions of energy (Sec. 2.1.1, Sec. 3.3.1)."""

    def __init__(self, materials, N, collision, transport_correction, p, alpha, t100):
        self.mats = [m if isinstance(m, Material) else Material.from_dict(m) for m in materials]
        self.N = N
        self.collision = collision
        self.etc = bool(transport_correction) and collision == BOLTZMANN
        # transport_correction == 2: delta-function corrected Fokker-Planck moments
        self.fp_delta = int(transport_correction) == 2 and collision != BOLTZMANN
        self.p = p
        self.alpha = alpha
        self.t100 = t100
        # unit-amplitude screened-Rutherford moments up to N+1 per material
        self._unit = []
        for m in self.mats:
            s, xi = screened_rutherford_unit_moments(m.screening, N + 1)
            self._unit.append((s, xi))

    def stopping_power(self, i, E):
        m = self.mats[i]
        return m.density * m.sp_ratio * stopping_power_water(E, self.p, self.alpha)

    def xi1(self, i, E):
        m = self.mats[i]
        return m.density * m.scatter_ratio * 0.5 * scattering_power_water(E, self.t100)

    def boltzmann_moments(self, i, E):
        """sigma_{i,l}(E) = 2 pi int P_l Sigma_{s;i} dmu for l = 0..N+1 (uncorrected)."""
        s, xi = self._unit[i]
        C = self.xi1(i, E) / xi
        return C * s

    def moments(self, i, E):
        """(G_{i,l} for l = 0..N, Sigma_{t,i}) as used in Eq. (discAngle).

        Boltzmann: G_l = sigma_l and Sigma_t = G_0 (Sec. 3.3.1), both shifted by
        -sigma_{N+1} under the extended transport correction.
        Fokker-Planck: G_l = -(xi_1/2) l (l+1), Sigma_t = 0 (Gamma_out = 0, Sec. 3.1); with the
        delta-function correction G_l = (xi_1/2) [(N+1)(N+2) - l(l+1)] and Sigma_t = G_0.
        """
        if self.collision == BOLTZMANN:
            sig = self.boltzmann_moments(i, E)
            G = sig[: self.N + 1].copy()
            if self.etc:
                G = G - sig[self.N + 1]
            return G, G[0]
        l = np.arange(self.N + 1, dtype=np.float64)
        xi = self.xi1(i, E)
        if self.fp_delta:
            G = 0.5 * xi * ((self.N + 1) * (self.N + 2) - l * (l + 1))
            return G, G[0]
        return -0.5 * xi * l * (l + 1), 0.0

    def self_scatter(self, i, E):
        """G_{i,l} - Sigma_{t,i}: the collided self-scattering eigenvalue per degree."""
        G, St = self.moments(i, E)
        return G - St

    def inscatter(self, i, E):
        """G_{i,l}: the in-scattering moments applied to the uncollided flux."""
        return self.moments(i, E)[0]

    def sigma_t(self, i, E):
        """Uncollided removal Sigma_{t,i} (Gamma_out, Sec. 3.1); E may be an array.

        Boltzmann: Sigma_t = G_0 = sigma_0 (minus sigma_{N+1} under the correction);
        Fokker-Planck: 0, or (xi_1/2)(N+1)(N+2) with the delta-function correction.
        """
        E = _num(E)
        if self.collision != BOLTZMANN:
            if self.fp_delta:
                return 0.5 * self.xi1(i, E) * (self.N + 1) * (self.N + 2)
            return np.zeros_like(E)
        s, xi = self._unit[i]
        C = self.xi1(i, E) / xi
        g0 = s[0] - (s[self.N + 1] if self.etc else 0.0)
        return C * g0
