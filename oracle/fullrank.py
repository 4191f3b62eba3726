"""Full-rank solve of the collided equation (oracle; test infrastructure only).

Sec. 3.3.2 semi-discrete system u' = F_S(u) + G(t, u) (Eq. streamscattsplit) with
u in R^{n x m}, split by first-order Lie splitting (Sec. 3.3.3) into streaming then
scattering; the full-rank method uses the same discretisation and integrators as
the low-rank one (Sec. 4): RK4 for streaming, implicit Euler for collided
self-scattering, explicit Euler for the first-collision source.

Reading of F_S (the paper's pairing of D^+ with Lambda^+ is downwind and
unstable; see tests/test_oracle_grid.py::test_literal_pairing_is_unstable):
  F_S(t, u) = sum_d [ D^-_d (S(t)^-1 u) A^+_d + D^+_d (S(t)^-1 u) A^-_d ],
  A^{+/-}_d = V_d Lambda^{+/-}_d V_d^T.
Collided scattering (Eq. discAngle, Sec. 3.3.3 step 1) for each cell x and moment p:
  u <- u / (1 - dE sum_i w_i(x)/S(x,E_{k+1}) (G_{i,l(p)} - Sigma_{t,i})).
Source (Sec. 3.3.3 steps 2-4, Eq. discAngle last term):
  u <- u + dE sum_i diag(w_i psi_u) 1 (G_i m(Omega_in))^T.
Dose (reading; the paper plots deposited energy without a formula): after each
step e(x) += dE sqrt(4 pi) u(x, 0), plus the uncollided deposit of the ray tracer.
"""
from __future__ import annotations

import math

import numpy as np

from . import angular
from .grid import apply_D

SQRT4PI = math.sqrt(4.0 * math.pi)


def rk4(f, t0, y0, h_total, nsub):
    """Classic fourth-order Runge-Kutta with nsub equal sub-steps."""
    h = h_total / nsub
    y = y0
    t = t0
    for _ in range(nsub):
        k1 = f(t, y)
        k2 = f(t + 0.5 * h, y + 0.5 * h * k1)
        k3 = f(t + 0.5 * h, y + 0.5 * h * k2)
        k4 = f(t + h, y + h * k3)
        y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        t = t + h
    return y


def streaming_rhs(prob, t, u):
    """F_S(t, u) of Eq. streamscattsplit (upwind reading)."""
    S = prob.stopping(prob.energy_at(t))
    Y = u / S[:, None]
    out = np.zeros_like(u)
    for d in prob.dirs:
        out += apply_D(Y, prob.dims, d, -1, prob.delta[d]) @ prob.ang.Ap[d]
        out += apply_D(Y, prob.dims, d, +1, prob.delta[d]) @ prob.ang.Am[d]
    return out


def scatter_factor(prob, k):
    """(n, m) array of dE * sum_i w_i/S (G_{i,l(p)} - Sigma_{t,i}) at E_{k+1}."""
    S = prob.stopping(prob.E[k + 1])
    g = prob.scatter_coefficients(k)           # (M, N+1)
    coef = np.zeros((prob.n, prob.m))
    for i in range(prob.M):
        coef += (prob.w[i] / S)[:, None] * g[i][prob.degree][None, :]
    return prob.h * coef


def source_factors(prob, k, psi_k, omega):
    """Rank-M factors of the first-collision source: Q = A B^T.

    A[:, i] = w_i(x) psi_u(x, k) (bin-averaged uncollided fluence),
    B[:, i] = G_{i,l(p)}(E_{k+1/2}) m_p(Omega_in).
    """
    A = prob.w.T * psi_k[:, None]                       # (n, M)
    G = prob.inscatter_coefficients(k)                  # (M, N+1)
    mo = angular.real_sh_dir(prob.N, omega)             # (m,)
    B = (G[:, prob.degree] * mo[None, :]).T             # (m, M)
    return A, B


def solve(prob, sources, n_steps=None, u0=None):
    """Full-rank run. ``sources``: list of (psi (K, n), e_u (n,), omega).

    ``u0`` is the collided state at E_max (zero, Sec. 3.3, unless given).
    Returns dict(dose, dose_collided, u).
    """
    K = prob.K if n_steps is None else n_steps
    u = np.zeros((prob.n, prob.m)) if u0 is None else np.array(u0, dtype=np.float64)
    e_c = np.zeros(prob.n)
    for k in range(K):
        t0 = k * prob.h
        u = rk4(lambda t, y: streaming_rhs(prob, t, y), t0, u, prob.h, prob.n_sub(k))
        u = u / (1.0 - scatter_factor(prob, k))
        for psi, _, omega in sources:
            if np.any(psi[k] != 0.0):
                A, B = source_factors(prob, k, psi[k], omega)
                u = u + prob.h * (A @ B.T)
        e_c += prob.h * SQRT4PI * u[:, 0]
    e_u = sum(src[1] for src in sources) if sources else np.zeros(prob.n)
    return dict(dose=e_c + e_u, dose_collided=e_c, u=u)
