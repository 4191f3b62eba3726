"""Discrete adjoint of the full-rank solve (oracle; test infrastructure only).

The paper gives the forward method only. Gradients of a loss L(e) of the deposited
energy e(x) (``fullrank.solve``: collided dose plus the uncollided deposit of every
beam) are defined here as the exact derivatives of that discrete forward map, taken
by reverse-mode differentiation of its steps in reverse order:

* with respect to each beam weight beta_b: the forward solve is linear in the
  sources and every source is linear in its beam weight (Sec. 3.2: the ray weights
  carry it), so dL/dbeta_b = <dL/de, e_b> with e_b the deposit of beam b at unit
  weight (the plain definition, one unit-weight solve per beam);
* with respect to the mixture weights w_i(x) (Sec. 2.1, Eq. mixXS), which enter
  the streaming through S(x, E) = sum_i w_i S_i(E), the collided self-scattering
  through w_i / S, the first-collision source through A_i = w_i psi_u, and the
  uncollided ray trace through S and Sigma_t.

Forward step k (``fullrank.solve``):  a = RK4^{n_sub}_{F_S}(u_k);  b = a / (1 - F_k);
u_{k+1} = b + dE sum_b beta_b A_b B_b^T;  e += dE sqrt(4 pi) u_{k+1}[:, 0].
Reverse step with ubar = dL/du_{k+1}:
  ubar[:, 0] += dE sqrt(4 pi) dL/de;
  source:  Abar_b = dE beta_b ubar B_b;  dw_i += Abar_b[:, i] psi_b;  dpsi_b += sum_i Abar_b[:, i] w_i;
  scatter: Fbar = ubar a / (1 - F)^2;  ubar <- ubar / (1 - F);
           dF/dw_i(x) = dE g_i(l) / S(x) - F S_i / S(x)  (S, g at E_{k+1});
  streaming: the transposed RK4 sub-steps in reverse order; for a stage f(t, z) = F_S(t, z)
           with adjoint kbar: zbar = F_S(t)^T kbar = S^-1 sum_d [(D^-_d)^T kbar (A^+_d)^T
           + (D^+_d)^T kbar (A^-_d)^T] and dL/dS(x) = -S(x)^-1 sum_p zbar(x, p) z(x, p),
           dS(x)/dw_i(x) = S_i(E_t).
The ray-trace part uses ``raytrace.trace_vjp`` (complex step) with dL/dpsi_b and
dL/de_{u,b} = beta_b dL/de. The sub-step count n_sub (a piecewise-constant function of
min_x S) is held fixed.

Pins (tests/test_oracle_adjoint.py): the transposed operators against the transposes of
assembled matrices and the adjoint identity <ybar, F y> = <F^T ybar, y>; the complete
gradient against central finite differences of ``fullrank.solve`` (exact up to
round-off for the beam weights of a quadratic loss, second order in the step for w).
"""
from __future__ import annotations

import numpy as np

from . import raytrace
from .fullrank import SQRT4PI, rk4, scatter_factor, source_factors, streaming_rhs
from .grid import apply_DT


def unit_sources(prob, beams):
    """(psi (K, n), e_u (n,), omega, beta) per beam, traced at unit weight."""
    out = []
    for b in beams:
        bu = dict(b)
        bu["weight"] = 1.0
        r = raytrace.trace(prob, bu)
        d = np.asarray(b["dir"], dtype=np.float64)
        out.append((r.psi, r.e_u, d / np.linalg.norm(d), float(b.get("weight", 1.0))))
    return out


def streaming_rhs_T(prob, t, ybar):
    """Transpose of the linear map y -> F_S(t, y) (upwind reading of Eq. streamscattsplit)."""
    S = prob.stopping(prob.energy_at(t))
    out = np.zeros_like(ybar)
    for d in prob.dirs:
        out += apply_DT(ybar @ prob.ang.Ap[d].T, prob.dims, d, -1, prob.delta[d])
        out += apply_DT(ybar @ prob.ang.Am[d].T, prob.dims, d, +1, prob.delta[d])
    return out / S[:, None]


def _stage_dw(prob, t, zbar, z):
    """d<kbar, F_S(t, z)>/dw_i(x) given zbar = F_S(t)^T kbar: -S_i(E) zbar(x,:).z(x,:) / S(x)."""
    E = prob.energy_at(t)
    S = prob.stopping(E)
    dS = -np.sum(zbar * z, axis=1) / S
    return np.array([prob.phys.stopping_power(i, E) * dS for i in range(prob.M)])


def rk4_vjp(prob, t0, y0, h_total, nsub, ybar):
    """Reverse of ``fullrank.rk4`` applied to F_S: returns (dL/dy0, dL/dw (M, n))."""
    h = h_total / nsub
    starts = [y0]
    for s in range(nsub):
        starts.append(rk4(lambda t, y: streaming_rhs(prob, t, y), t0 + s * h, starts[-1], h, 1))
    dw = np.zeros((prob.M, prob.n))
    for s in reversed(range(nsub)):
        t = t0 + s * h
        y = starts[s]
        f = lambda tt, z: streaming_rhs(prob, tt, z)
        k1 = f(t, y)
        z2 = y + 0.5 * h * k1
        k2 = f(t + 0.5 * h, z2)
        z3 = y + 0.5 * h * k2
        k3 = f(t + 0.5 * h, z3)
        z4 = y + h * k3
        yb = ybar.copy()
        k1b = (h / 6.0) * ybar
        k2b = (h / 3.0) * ybar
        k3b = (h / 3.0) * ybar
        k4b = (h / 6.0) * ybar
        # k4 = f(t + h, z4), z4 = y + h k3
        zb = streaming_rhs_T(prob, t + h, k4b)
        dw += _stage_dw(prob, t + h, zb, z4)
        yb += zb
        k3b = k3b + h * zb
        # k3 = f(t + h/2, z3), z3 = y + h/2 k2
        zb = streaming_rhs_T(prob, t + 0.5 * h, k3b)
        dw += _stage_dw(prob, t + 0.5 * h, zb, z3)
        yb += zb
        k2b = k2b + 0.5 * h * zb
        # k2 = f(t + h/2, z2), z2 = y + h/2 k1
        zb = streaming_rhs_T(prob, t + 0.5 * h, k2b)
        dw += _stage_dw(prob, t + 0.5 * h, zb, z2)
        yb += zb
        k1b = k1b + 0.5 * h * zb
        # k1 = f(t, y)
        zb = streaming_rhs_T(prob, t, k1b)
        dw += _stage_dw(prob, t, zb, y)
        yb += zb
        ybar = yb
    return ybar, dw


def scatter_dF_dw(prob, k):
    """(M, n, m): dF(x, p)/dw_i(x) for F = scatter_factor(prob, k)."""
    E = prob.E[k + 1]
    S = prob.stopping(E)
    g = prob.scatter_coefficients(k)                       # (M, N+1)
    F = scatter_factor(prob, k)
    out = np.empty((prob.M, prob.n, prob.m))
    for i in range(prob.M):
        out[i] = prob.h * g[i][prob.degree][None, :] / S[:, None] \
            - F * (prob.phys.stopping_power(i, E) / S)[:, None]
    return out


def gradient(prob, beams, dL_de, n_steps=None, with_raytrace=True):
    """Gradient of L at the forward solve of ``beams`` for dL/de = ``dL_de`` (n,).

    Returns dict(dbeta (B,), dw (M, n), dpsi [per beam (K, n)], dw_trace (M, n)).
    """
    K = prob.K if n_steps is None else n_steps
    src = unit_sources(prob, beams)
    g_e = np.asarray(dL_de, dtype=np.float64)
    # beam weights: one unit-weight forward solve per beam
    from .fullrank import solve as fr_solve
    dbeta = np.array([float(g_e @ fr_solve(prob, [(p, e, o)], n_steps=K)["dose"]) for p, e, o, _ in src])
    # forward, storing the state before every step
    us = []
    u = np.zeros((prob.n, prob.m))
    for k in range(K):
        us.append(u)
        a = rk4(lambda t, y: streaming_rhs(prob, t, y), k * prob.h, u, prob.h, prob.n_sub(k))
        b = a / (1.0 - scatter_factor(prob, k))
        for psi, _, om, beta in src:
            if np.any(psi[k] != 0.0):
                A, B = source_factors(prob, k, psi[k], om)
                b = b + prob.h * beta * (A @ B.T)
        u = b
    # reverse sweep
    dw = np.zeros((prob.M, prob.n))
    dpsi = [np.zeros((prob.K, prob.n)) for _ in src]
    ubar = np.zeros((prob.n, prob.m))
    for k in reversed(range(K)):
        ubar[:, 0] += prob.h * SQRT4PI * g_e
        for j, (psi, _, om, beta) in enumerate(src):
            if np.any(psi[k] != 0.0):
                _, B = source_factors(prob, k, psi[k], om)
                Abar = prob.h * beta * (ubar @ B)                     # (n, M)
                for i in range(prob.M):
                    dw[i] += Abar[:, i] * psi[k]
                dpsi[j][k] += np.sum(Abar * prob.w.T, axis=1)
        a = rk4(lambda t, y: streaming_rhs(prob, t, y), k * prob.h, us[k], prob.h, prob.n_sub(k))
        F = scatter_factor(prob, k)
        Fbar = ubar * a / (1.0 - F) ** 2
        dw += np.einsum("xp,ixp->ix", Fbar, scatter_dF_dw(prob, k))
        ubar = ubar / (1.0 - F)
        ubar, dws = rk4_vjp(prob, k * prob.h, us[k], prob.h, prob.n_sub(k), ubar)
        dw += dws
    dw_trace = np.zeros((prob.M, prob.n))
    if with_raytrace:
        for j, b in enumerate(beams):
            bu = dict(b)
            bu["weight"] = 1.0
            dw_trace += raytrace.trace_vjp(prob, bu, dpsi[j], src[j][3] * g_e)
    return dict(dbeta=dbeta, dw=dw + dw_trace, dw_collided=dw, dw_trace=dw_trace, dpsi=dpsi)


def loss_and_dose(prob, beams, n_steps=None):
    """Forward deposit e(x) of ``fullrank.solve`` with the beams traced by ``raytrace.trace``."""
    from .fullrank import solve as fr_solve
    srcs = []
    for b in beams:
        r = raytrace.trace(prob, b)
        d = np.asarray(b["dir"], dtype=np.float64)
        srcs.append((r.psi, r.e_u, d / np.linalg.norm(d)))
    return fr_solve(prob, srcs, n_steps=n_steps)["dose"]


def finite_difference(prob_factory, beams, w, loss_fn, i, x, rel=1e-6):
    """Central difference of loss_fn(e(w)) in w_i(x) (for the pins); prob_factory(w) -> Problem."""
    eps = rel * max(abs(w[i, x]), 1e-3)
    wp = w.copy()
    wp[i, x] += eps
    wm = w.copy()
    wm[i, x] -= eps
    return (loss_fn(loss_and_dose(prob_factory(wp), beams)) - loss_fn(loss_and_dose(prob_factory(wm), beams))) \
        / (2.0 * eps)
