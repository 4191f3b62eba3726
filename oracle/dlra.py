"""Low-rank energy step: augmented BUG integrator (oracle; test infrastructure only).

The collided moments are kept as u = X S W^T with X (n x r) and W (m x r)
orthonormal (Sec. 2.2). One energy step k -> k+1 (Sec. 3.3.3):

1. Streaming, Eq. split-streaming, with the augmented BUG integrator of Sec. 2.2
   (Eq. KLS) and RK4 for every time update:
     K' = F_S(t, K W0^T) W0,  K(t0) = X0 S0
     L' = F_S(t, X0 L^T)^T X0, L(t0) = W0 S0^T
     X^ spans [K(t1), X0], W^ spans [L(t1), W0]
     S' = X^^T F_S(t, X^ S W^^T) W^, S(t0) = (X^^T X0) S0 (W0^T W^)
   then truncation of the SVD of S(t1) (Sec. 2.2).
2. Collided self-scattering, projector-splitting L-step with implicit Euler
   (Sec. 3.3.3 step 1): L' = sum_i M_i(t) L (G_i - Sigma_{t,i}),
   M_i = X^T w_i S^-1 X, L(t0) = S W^T; then QR of L(t1)^T = W~ S~^T.
3. First-collision source, augmented BUG K/L/S steps with explicit Euler
   (Sec. 3.3.3 steps 2-4), then truncation.

Readings (the paper is silent or ambiguous; the GPU path takes the same):
* The source term is rank M per beam, Q = A B^T (fullrank.source_factors). The
  K-step and L-step of step 3 give X^ = span[X, (I - X X^T) A (B^T W~)] and
  W^ = span[W~, (I - W~ W~^T) B (A^T X)]; whenever B^T W~ and A^T X have full
  column rank these equal span[X, A] and span[W~, B], which is what is used. This
  also covers the rank-0 start u(E_max) = 0, where the literal K-step is empty.
  The S-step with explicit Euler is then S1 = X^^T (X S~ W~^T + dE A B^T) W^.
* Steps 2-4 start from the post-collision state X S~ W~^T (the paper's
  W~^{1/2,T} W^ has mismatched dimensions as printed).
* Bases are augmented rank-revealingly: directions of (I - X X^T) K whose
  singular values are below drop_tol * ||K||_2 are dropped (a square full-rank
  problem therefore reproduces the full-rank solve to round-off).
* Truncation rule: FIXED keeps min(r, #sigma > 1e-14 sigma_1); ADAPTIVE keeps the
  smallest r1 with sum_{i > r1} sigma_i <= tol * ||sigma||_2, clamped to
  [1, r_max]; SCHEDULE replays given ranks. No cut inside a cluster of
  singular values closer than cluster_tol * sigma_1 (the cut moves down, or up
  if it would reach zero), so symmetric pairs stay together.
* Dose: e(x) += dE sqrt(4 pi) (X S W^T)(x, 0) after each step.
"""
from __future__ import annotations

import math

import numpy as np

from .fullrank import SQRT4PI, rk4
from .grid import apply_D
from .problem import ADAPTIVE, FIXED, SCHEDULE


def augment(X, K, drop_tol=1e-12):
    """Orthonormal basis of span[X, K] whose first columns are X (rank-revealing)."""
    n = X.shape[0]
    if K.shape[1] == 0:
        return X.copy()
    scale = np.linalg.norm(K, 2)
    if scale == 0.0:
        return X.copy()
    R = K - X @ (X.T @ K)
    R = R - X @ (X.T @ R)
    U, s, _ = np.linalg.svd(R, full_matrices=False)
    keep = s > drop_tol * scale
    return np.hstack([X, U[:, keep]]) if X.shape[1] else U[:, keep].reshape(n, -1)


def choose_rank(s, mode, rank=None, tol=None, r_max=None, sched=None, cluster_tol=1e-10,
                nz_tol=1e-14):
    if s.size == 0 or s[0] <= 0.0:
        return 0
    if mode == SCHEDULE:
        return int(min(sched, s.size))
    nz = int(np.sum(s > nz_tol * s[0]))
    if mode == FIXED:
        r1 = min(int(rank), nz)
    else:
        thr = tol * np.linalg.norm(s)
        tails = np.concatenate([np.cumsum(s[::-1])[::-1], [0.0]])  # tails[r] = sum s[r:]
        r1 = int(np.argmax(tails <= thr))
        r1 = max(1, min(r1, int(r_max), nz))
    r0 = r1
    while 0 < r1 < s.size and s[r1 - 1] - s[r1] <= cluster_tol * s[0]:
        r1 -= 1
    if r1 == 0:
        r1 = r0
        while r1 < s.size and s[r1 - 1] - s[r1] <= cluster_tol * s[0]:
            r1 += 1
    return r1


def truncate(Xh, Sh, Wh, r1):
    P, s, Qt = np.linalg.svd(Sh)
    return Xh @ P[:, :r1], np.diag(s[:r1]), Wh @ Qt[:r1].T, s


class RankControl:
    def __init__(self, mode=FIXED, rank=5, tol=1e-3, r_max=64, schedule=None, cluster_tol=1e-10):
        self.mode = mode
        self.rank = rank
        self.tol = tol
        self.r_max = r_max
        self.schedule = schedule      # array (K, 2): ranks after streaming / source, -1 = none
        self.cluster_tol = cluster_tol

    def pick(self, s, k, event):
        sched = None
        if self.mode == SCHEDULE:
            sched = int(self.schedule[k][event])
        return choose_rank(s, self.mode, self.rank, self.tol, self.r_max, sched, self.cluster_tol)


def streaming_operators(prob, t, Xa, Xb):
    """X_a^T D^{+/-}_d S(t)^-1 X_b for each streaming direction d."""
    S = prob.stopping(prob.energy_at(t))
    Y = Xb / S[:, None]
    Gp, Gm = {}, {}
    for d in prob.dirs:
        Gp[d] = Xa.T @ apply_D(Y, prob.dims, d, +1, prob.delta[d])
        Gm[d] = Xa.T @ apply_D(Y, prob.dims, d, -1, prob.delta[d])
    return Gp, Gm


def streaming_bug(prob, X, S, W, k, drop_tol=1e-12):
    """Step 1 before truncation: returns (X^, S(t1), W^, K1, L1)."""
    h = prob.h
    t0 = k * h
    nsub = prob.n_sub(k)
    ang = prob.ang
    Pp = {d: W.T @ ang.Ap[d] @ W for d in prob.dirs}
    Pm = {d: W.T @ ang.Am[d] @ W for d in prob.dirs}

    def fK(t, K):
        Sx = prob.stopping(prob.energy_at(t))
        Y = K / Sx[:, None]
        out = np.zeros_like(K)
        for d in prob.dirs:
            out += apply_D(Y, prob.dims, d, -1, prob.delta[d]) @ Pp[d]
            out += apply_D(Y, prob.dims, d, +1, prob.delta[d]) @ Pm[d]
        return out

    def fL(t, L):
        Gp, Gm = streaming_operators(prob, t, X, X)
        out = np.zeros_like(L)
        for d in prob.dirs:
            out += ang.Ap[d] @ L @ Gm[d].T + ang.Am[d] @ L @ Gp[d].T
        return out

    K1 = rk4(fK, t0, X @ S, h, nsub)
    L1 = rk4(fL, t0, W @ S.T, h, nsub)
    Xh = augment(X, K1, drop_tol)
    Wh = augment(W, L1, drop_tol)
    Pph = {d: Wh.T @ ang.Ap[d] @ Wh for d in prob.dirs}
    Pmh = {d: Wh.T @ ang.Am[d] @ Wh for d in prob.dirs}

    def fS(t, Sh):
        Gp, Gm = streaming_operators(prob, t, Xh, Xh)
        out = np.zeros_like(Sh)
        for d in prob.dirs:
            out += Gm[d] @ Sh @ Pph[d] + Gp[d] @ Sh @ Pmh[d]
        return out

    S0 = (Xh.T @ X) @ S @ (W.T @ Wh)
    S1 = rk4(fS, t0, S0, h, nsub)
    return Xh, S1, Wh, K1, L1


def collided_scatter(prob, X, S, W, k):
    """Step 2: implicit-Euler L-step at E_{k+1}, then QR. Returns (X, S~, W~)."""
    r = X.shape[1]
    Sx = prob.stopping(prob.E[k + 1])
    g = prob.scatter_coefficients(k)             # (M, N+1)
    Mi = [X.T @ (X * (prob.w[i] / Sx)[:, None]) for i in range(prob.M)]
    L0 = S @ W.T                                  # (r, m)
    L1 = np.empty_like(L0)
    I = np.eye(r)
    for p in range(prob.m):
        l = prob.degree[p]
        A = I - prob.h * sum(g[i, l] * Mi[i] for i in range(prob.M))
        L1[:, p] = np.linalg.solve(A, L0[:, p])
    Q, R = np.linalg.qr(L1.T)
    return X, R.T, Q


def source_bug(prob, X, S, W, A, B, drop_tol=1e-12):
    """Steps 2-4 (explicit Euler) before truncation: returns (X^, S1, W^)."""
    Xh = augment(X, A, drop_tol)
    Wh = augment(W, B, drop_tol)
    S1 = (Xh.T @ X) @ S @ (W.T @ Wh) + prob.h * (Xh.T @ A) @ (B.T @ Wh)
    return Xh, S1, Wh


class State:
    def __init__(self, n, m):
        self.X = np.zeros((n, 0))
        self.S = np.zeros((0, 0))
        self.W = np.zeros((m, 0))

    @property
    def r(self):
        return self.X.shape[1]

    def u(self):
        return self.X @ self.S @ self.W.T

    def moment0(self):
        return self.X @ (self.S @ self.W[0, :]) if self.r else np.zeros(self.X.shape[0])


def step(prob, st: State, k, sources, rc: RankControl, drop_tol=1e-12, log=None):
    """One full energy step k -> k+1 on state ``st`` (in place)."""
    from .fullrank import source_factors
    ranks = [-1, -1]
    if st.r > 0:
        Xh, Sh, Wh, _, _ = streaming_bug(prob, st.X, st.S, st.W, k, drop_tol)
        _, s, _ = np.linalg.svd(Sh) if Sh.size else (None, np.zeros(0), None)
        r1 = rc.pick(s, k, 0)
        st.X, st.S, st.W, _ = truncate(Xh, Sh, Wh, r1)
        ranks[0] = r1
        if r1 > 0:
            st.X, st.S, st.W = collided_scatter(prob, st.X, st.S, st.W, k)
    active = [(psi, om) for psi, _, om in sources if np.any(psi[k] != 0.0)]
    if active:
        As, Bs = [], []
        for psi, om in active:
            A, B = source_factors(prob, k, psi[k], om)
            As.append(A)
            Bs.append(B)
        A = np.hstack(As)
        B = np.hstack(Bs)
        Xh, Sh, Wh = source_bug(prob, st.X, st.S, st.W, A, B, drop_tol)
        _, s, _ = np.linalg.svd(Sh) if Sh.size else (None, np.zeros(0), None)
        r1 = rc.pick(s, k, 1)
        st.X, st.S, st.W, _ = truncate(Xh, Sh, Wh, r1)
        ranks[1] = r1
    if log is not None:
        log.append(ranks)
    return ranks


def solve(prob, sources, rc: RankControl, n_steps=None, drop_tol=1e-12, state=None):
    """Low-rank run from ``state`` (rank 0 at E_max unless given).

    Returns dict(dose, dose_collided, state, ranks (K, 2)).
    """
    K = prob.K if n_steps is None else n_steps
    st = State(prob.n, prob.m) if state is None else state
    e_c = np.zeros(prob.n)
    log = []
    for k in range(K):
        step(prob, st, k, sources, rc, drop_tol, log)
        e_c += prob.h * SQRT4PI * st.moment0()
    e_u = sum(src[1] for src in sources) if sources else np.zeros(prob.n)
    return dict(dose=e_c + e_u, dose_collided=e_c, state=st, ranks=np.array(log, dtype=np.int64))
