"""One transport problem: grid, energy grid, mixture coefficients (oracle; test infrastructure only).

Sec. 2.1 (mixture rule, Eq. mixXS and Eq. finalContinuous), Sec. 3.3 (pseudo-time
t = E_max - E): the collided equation is advanced on a uniform energy grid
E_0 = E_max > E_1 > ... > E_K = E_min with Delta t = Delta E.

Readings where the paper is silent (each listed in the design notes):
* the mixture stopping power S(x, E) = sum_i w_i(x) S_i(E) (Bragg additivity);
* streaming sub-cycling: the paper gives no stability rule; each energy step's
  streaming ODEs are integrated with n_sub RK4 sub-steps,
  n_sub = max(1, ceil(dE * sum_d lam_max(A_d)/delta_d / (min_x S(x, E_k) * cfl))),
  the sum running over the streaming directions (x, z in a 2-D x-z slab);
* coefficient energies: streaming at the RK4 stage energies, collided
  self-scattering at E_{k+1} (implicit Euler), in-scattering at E_{k+1/2}.
"""
from __future__ import annotations

import math

import numpy as np

from . import angular, physics

FIXED, ADAPTIVE, SCHEDULE = 0, 1, 2

DEFAULTS = dict(
    transport_correction=1,
    rank_mode=FIXED,
    rank=5,
    rank_max=64,
    trunc_tol=1e-3,
    cfl=0.6,
    bk_p=1.77,
    bk_alpha=0.0022,
    t100=1.72e-4,
)


def _collision_code(c):
    if isinstance(c, str):
        return physics.BOLTZMANN if c.lower().startswith("b") else physics.FOKKER_PLANCK
    return int(c)


class Problem:
    def __init__(self, cfg: dict, materials, w: np.ndarray, angular_tables=None):
        c = dict(DEFAULTS)
        c.update(cfg)
        self.cfg = c
        self.nx, self.ny, self.nz = int(c["nx"]), int(c["ny"]), int(c["nz"])
        self.dx, self.dy, self.dz = float(c["dx"]), float(c["dy"]), float(c["dz"])
        self.two_d = self.ny == 1 and self.dy == 0.0
        self.dims = (self.nx, self.ny, self.nz)
        self.n = self.nx * self.ny * self.nz
        self.N = int(c["N"])
        self.m = angular.n_moments(self.N)
        self.collision = _collision_code(c["collision"])
        self.ang = angular_tables if angular_tables is not None else angular.AngularTables(self.N)
        self.phys = physics.PhysicsTables(materials, self.N, self.collision, c["transport_correction"],
                                          c["bk_p"], c["bk_alpha"], c["t100"])
        self.M = len(self.phys.mats)
        w = np.asarray(w, dtype=np.float64)
        self.w = w.reshape(self.M, self.n)
        self.e_max, self.e_min = float(c["e_max"]), float(c["e_min"])
        self.K = int(c["n_steps"])
        self.h = (self.e_max - self.e_min) / self.K
        self.E = self.e_max - self.h * np.arange(self.K + 1)
        # streaming directions and spacings
        self.dirs = [0, 2] if self.two_d else [0, 1, 2]
        self.delta = {0: self.dx, 1: self.dy, 2: self.dz}
        self.volume = self.dx * self.dz * (1.0 if self.two_d else self.dy)
        self.degree = self.ang.degree

    # -- mixture coefficients (Eq. mixXS) ---------------------------------
    def stopping(self, E: float) -> np.ndarray:
        """S(x, E) = sum_i w_i(x) S_i(E), shape (n,)."""
        out = np.zeros(self.n)
        for i in range(self.M):
            out += self.w[i] * self.phys.stopping_power(i, E)
        return out

    def sigma_t(self, E: float) -> np.ndarray:
        """Sigma_t(x, E) = sum_i w_i Sigma_{t,i}(E), shape (n,)."""
        out = np.zeros(self.n)
        for i in range(self.M):
            out += self.w[i] * self.phys.sigma_t(i, E)
        return out

    def energy_at(self, t: float) -> float:
        """Pseudo-time t = E_max - E (Sec. 3.3)."""
        return self.e_max - t

    def n_sub(self, k: int) -> int:
        lam = sum(self.ang.lam_max[d] / self.delta[d] for d in self.dirs)
        smin = float(np.min(self.stopping(self.E[k])))
        nu = self.h * lam / (smin * self.cfg["cfl"])
        return max(1, int(math.ceil(nu - 1e-9)))

    def scatter_coefficients(self, k: int) -> np.ndarray:
        """(M, N+1): G_{i,l} - Sigma_{t,i} at E_{k+1} (collided self-scattering)."""
        E = self.E[k + 1]
        return np.array([self.phys.self_scatter(i, E) for i in range(self.M)])

    def inscatter_coefficients(self, k: int) -> np.ndarray:
        """(M, N+1): G_{i,l} at E_{k+1/2} (in-scattering of the uncollided flux)."""
        E = 0.5 * (self.E[k] + self.E[k + 1])
        return np.array([self.phys.inscatter(i, E) for i in range(self.M)])
