"""Low-rank reverse sweep: gradients of the low-rank solve (oracle; test infrastructure only).

The paper gives no adjoint. The exact gradient of the full-rank discrete solve is
``adjoint.gradient`` (a plain definition: reverse-mode differentiation). This module
writes out, step by step and with plain numpy, the low-rank approximation of that
reverse sweep which the library runs, so that the library can be compared with it
at round-off (its distance to ``adjoint.gradient`` is an approximation error, pinned
by convergence):

* forward: one independent low-rank state per beam at unit weight (``dlra``), the
  state at the start of every energy step kept;
* the adjoint state mu = X S W^T of dL/du starts at rank 0 after the last step; reverse
  step k: mu += dE sqrt(4 pi) (dL/de) e_0^T (the dose reads the l = 0 moment; a rank-1
  explicit source step, ``dlra.source_bug``, then truncation); the source gradients read
  mu; then the collision step of ``dlra.collided_scatter`` (the factor 1/(1 - F) is
  diagonal, so it is its own transpose) and a streaming BUG step with the transposed
  operator F_S^T(t) mu = S^-1 sum_d [(D^-_d)^T mu A^+_d + (D^+_d)^T mu A^-_d] (K-, L- and
  S-steps with the transposes of the Galerkin operators, then truncation);
* gradient terms with the forward state u_k of each beam b (weight beta_b):
  source: dL/dw_i(x) += dE beta_b psi_b(x) (mu B_{b,i})(x), dL/dpsi_b(x) = dE beta_b
  sum_i w_i(x) (mu B_{b,i})(x); collision: D(x, p) = alpha(x, p) b_k(x, p) (alpha = mu after
  the adjoint collision step, b_k = forward state after collision), dL/dw_i(x) +=
  beta_b sum_p D dF/dw_i; streaming: each RK4 sub-step of y' = c(t) L y with L y =
  sum_d D^(-/+)_d(rho_s^-1 y) A^(+/-)_d is the polynomial 1 + b_1 L (1 + b_2 L (1 + b_3 L
  (1 + b_4 L))) (the Taylor coefficients a_i of classic RK4 for a scalar-varying linear
  ODE, b_1 = a_1, b_{i+1} = a_{i+1}/a_i); with z_3..z_0 the Horner stage inputs of the
  forward K-step and lam_3 = b_1 L^T mu, lam_{i-1} = b_{5-i} L^T lam_i their adjoints (the
  adjoint K-step, run over the sub-steps in reverse order),
  dL/d rho_s(x) -= beta_b sum_{sub-steps, i} <rho_s^-1 z_i(x,:), lam_i(x,:)>;
  the uncollided part is ``raytrace.trace_vjp``; dL/dw_i = direct terms + rho_i s_i dL/d rho_s.

Pins (tests/test_oracle_adjoint.py): with one energy step every low-rank step is exact
and the gradient equals ``adjoint.gradient``; the Horner K-step equals the classic RK4
K-step of ``dlra.streaming_bug``; the gradient converges to ``adjoint.gradient`` as the
energy step shrinks.
"""
from __future__ import annotations

import math

import numpy as np

from . import adjoint, raytrace
from . import dlra as DL
from .fullrank import rk4, scatter_factor, source_factors
from .grid import apply_D, apply_DT


def horner_coefficients(prob, Ea, hs):
    """(b_4, b_3, b_2, b_1) of one RK4 sub-step from energy Ea for y' = L y / S_w(E(t)).

    Classic RK4 with c_1 = c(t), c_2 = c(t + h/2), c_4 = c(t + h) applied to the linear
    ODE gives y_1 = (1 + a_1 L + a_2 L^2 + a_3 L^3 + a_4 L^4) y_0 with a_1 = h (c_1 + 4 c_2
    + c_4)/6, a_2 = h^2 (c_1 c_2 + c_2^2 + c_2 c_4)/6, a_3 = h^3 (c_1 c_2^2 + c_2^2 c_4)/12,
    a_4 = h^4 c_1 c_2^2 c_4 / 24.
    """
    sw = lambda E: float(prob.phys.stopping_power(0, E)) / (prob.phys.mats[0].density * prob.phys.mats[0].sp_ratio)
    c1, c2, c4 = 1.0 / sw(Ea), 1.0 / sw(Ea - 0.5 * hs), 1.0 / sw(Ea - hs)
    a1 = hs * (c1 + 4 * c2 + c4) / 6.0
    a2 = hs ** 2 * (c1 * c2 + c2 * c2 + c2 * c4) / 6.0
    a3 = hs ** 3 * (c1 * c2 * c2 + c2 * c2 * c4) / 12.0
    a4 = hs ** 4 * c1 * c2 * c2 * c4 / 24.0
    return [a4 / a3, a3 / a2, a2 / a1, a1]


def rho_s(prob):
    """rho_s(x) = sum_i w_i rho_i s_i: S(x, E) = rho_s(x) S_w(E) (Eq. mixXS, separable)."""
    return sum(prob.w[i] * prob.phys.mats[i].density * prob.phys.mats[i].sp_ratio for i in range(prob.M))


def kstep(prob, X, S, W, k, transposed):
    """K-step of energy step k in Horner form. Forward: returns (K1, v) with v[4 j + i] the
    input rho_s^-1 z_i of stage i of sub-step j. Transposed: returns (K1, lam) with
    lam[4 j + i] the adjoint of z_i (sub-steps run in reverse order)."""
    g = rho_s(prob)
    Pp = {d: W.T @ prob.ang.Ap[d] @ W for d in prob.dirs}
    Pm = {d: W.T @ prob.ang.Am[d] @ W for d in prob.dirs}

    def L(Z):
        Y = Z / g[:, None]
        return sum(apply_D(Y, prob.dims, d, -1, prob.delta[d]) @ Pp[d]
                   + apply_D(Y, prob.dims, d, +1, prob.delta[d]) @ Pm[d] for d in prob.dirs)

    def LT(Z):
        return sum(apply_DT(Z @ Pp[d].T, prob.dims, d, -1, prob.delta[d])
                   + apply_DT(Z @ Pm[d].T, prob.dims, d, +1, prob.delta[d]) for d in prob.dirs) / g[:, None]

    ns = prob.n_sub(k)
    hs = prob.h / ns
    y = X @ S
    stages = [None] * (4 * ns)
    if not transposed:
        for j in range(ns):
            b = horner_coefficients(prob, prob.E[k] - j * hs, hs)
            z = y
            for i in range(4):
                stages[4 * j + i] = z / g[:, None]
                z = y + b[i] * L(z)
            y = z
    else:
        for j in reversed(range(ns)):
            b = horner_coefficients(prob, prob.E[k] - j * hs, hs)
            lam = y
            acc = y.copy()
            for i in reversed(range(4)):
                lam = b[i] * LT(lam)
                stages[4 * j + i] = lam
                acc = acc + lam
            y = acc
    return y, stages


def streaming(prob, X, S, W, k, transposed, rc, drop_tol=1e-12):
    """Augmented BUG streaming step (Sec. 2.2, Eq. KLS) of F_S or of its transpose, truncated.
    Returns (X, S, W, K-step stages)."""
    K1, stages = kstep(prob, X, S, W, k, transposed)
    ang = prob.ang
    t0 = k * prob.h
    ns = prob.n_sub(k)

    def fL(t, Lm):
        Gp, Gm = DL.streaming_operators(prob, t, X, X)
        if transposed:
            return sum(ang.Ap[d] @ Lm @ Gm[d] + ang.Am[d] @ Lm @ Gp[d] for d in prob.dirs)
        return sum(ang.Ap[d] @ Lm @ Gm[d].T + ang.Am[d] @ Lm @ Gp[d].T for d in prob.dirs)

    L1 = rk4(fL, t0, W @ S.T, prob.h, ns)
    Xh = DL.augment(X, K1, drop_tol)
    Wh = DL.augment(W, L1, drop_tol)
    Pph = {d: Wh.T @ ang.Ap[d] @ Wh for d in prob.dirs}
    Pmh = {d: Wh.T @ ang.Am[d] @ Wh for d in prob.dirs}

    def fS(t, Sh):
        Gp, Gm = DL.streaming_operators(prob, t, Xh, Xh)
        if transposed:
            return sum(Gm[d].T @ Sh @ Pph[d] + Gp[d].T @ Sh @ Pmh[d] for d in prob.dirs)
        return sum(Gm[d] @ Sh @ Pph[d] + Gp[d] @ Sh @ Pmh[d] for d in prob.dirs)

    S1 = rk4(fS, t0, (Xh.T @ X) @ S @ (W.T @ Wh), prob.h, ns)
    _, s, _ = np.linalg.svd(S1)
    Xn, Sn, Wn, _ = DL.truncate(Xh, S1, Wh, rc.pick(s, k, 0))
    return Xn, Sn, Wn, stages


def _truncated(rc, Xh, Sh, Wh, k, event):
    _, s, _ = np.linalg.svd(Sh)
    return DL.truncate(Xh, Sh, Wh, rc.pick(s, k, event))[:3]


def gradient(prob, beams, dL_de, rc, adjoint_rc=None, drop_tol=1e-12):
    """(dbeta (B,), dw (M, n)) of the low-rank solve of ``beams`` (rank control ``rc``)
    for dL/de = ``dL_de``; the adjoint state uses ``adjoint_rc`` (default ``rc``)."""
    arc = rc if adjoint_rc is None else adjoint_rc
    K, n, m, M = prob.K, prob.n, prob.m, prob.M
    g = np.asarray(dL_de, dtype=np.float64)
    src = adjoint.unit_sources(prob, beams)
    states, first, dbeta = [], [], []
    for psi, _, om, _ in src:
        X, S, W = np.zeros((n, 0)), np.zeros((0, 0)), np.zeros((m, 0))
        f = next((k for k in range(K) if np.any(psi[k] != 0.0)), -1)
        seq, e = [], np.zeros(n)
        for k in range(K):
            seq.append((X, S, W))
            if f >= 0 and k > f:
                Xh, Sh, Wh, _, _ = DL.streaming_bug(prob, X, S, W, k, drop_tol)
                X, S, W = _truncated(rc, Xh, Sh, Wh, k, 0)
                X, S, W = DL.collided_scatter(prob, X, S, W, k)
            if np.any(psi[k] != 0.0):
                A, B = source_factors(prob, k, psi[k], om)
                X, S, W = _truncated(rc, *DL.source_bug(prob, X, S, W, A, B, drop_tol), k, 1)
            e += prob.h * math.sqrt(4.0 * math.pi) * (X @ (S @ W[0, :]) if X.shape[1] else 0.0)
        states.append(seq)
        first.append(f)
        dbeta.append(float(g @ (e + src[len(dbeta)][1])))
    gr = rho_s(prob)
    cs = np.array([prob.phys.mats[i].density * prob.phys.mats[i].sp_ratio for i in range(M)])
    dw = np.zeros((M, n))
    grho = np.zeros(n)
    dpsi = [np.zeros((K, n)) for _ in src]
    mu = (np.zeros((n, 0)), np.zeros((0, 0)), np.zeros((m, 0)))
    e0 = np.zeros((m, 1))
    e0[0, 0] = math.sqrt(4.0 * math.pi)
    for k in reversed(range(K)):
        mu = _truncated(arc, *DL.source_bug(prob, *mu, g[:, None], e0, drop_tol), k, 1)
        U = mu[0] @ mu[1] @ mu[2].T
        for b, (psi, _, om, beta) in enumerate(src):
            if np.any(psi[k] != 0.0):
                _, B = source_factors(prob, k, psi[k], om)
                t = U @ B
                dw += prob.h * beta * (psi[k][:, None] * t).T
                dpsi[b][k] = prob.h * beta * np.sum(prob.w.T * t, axis=1)
        active = [first[b] >= 0 and k > first[b] for b in range(len(src))]
        if not any(active):
            continue
        alpha = DL.collided_scatter(prob, *mu, k)
        Xa, Sa, Wa, lam = streaming(prob, *alpha, k, True, arc, drop_tol)
        mu = (Xa, Sa, Wa)
        Ua = alpha[0] @ alpha[1] @ alpha[2].T
        F = scatter_factor(prob, k)
        E1 = prob.E[k + 1]
        Sw1 = float(prob.phys.stopping_power(0, E1)) / cs[0]
        coef = prob.scatter_coefficients(k)
        for b, (psi, _, om, beta) in enumerate(src):
            if not active[b]:
                continue
            X, S, W = states[b][k]
            _, v = kstep(prob, X, S, W, k, False)
            C = W.T @ alpha[2]
            for q in range(len(v)):
                grho -= beta * np.sum((v[q] @ C) * lam[q], axis=1)
            Xb, Sb, Wb, _ = streaming(prob, X, S, W, k, False, rc, drop_tol)
            Xb, Sb, Wb = DL.collided_scatter(prob, Xb, Sb, Wb, k)
            D = Ua * (Xb @ Sb @ Wb.T)
            for i in range(M):
                dw[i] += beta * np.sum(D * (prob.h * coef[i][prob.degree][None, :] / Sw1), axis=1) / gr
            grho -= beta * np.sum(D * F, axis=1) / gr
    dw += cs[:, None] * grho[None, :]
    for b, bm in enumerate(beams):
        bu = dict(bm)
        bu["weight"] = 1.0
        dw += raytrace.trace_vjp(prob, bu, dpsi[b], src[b][3] * g)
    return dict(dbeta=np.array(dbeta), dw=dw, dpsi=dpsi)
