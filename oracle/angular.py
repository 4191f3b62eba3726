"""Angular P_N tables (oracle; test infrastructure only).

Sec. 3.3.1 of the paper: the collided flux is expanded in real spherical
harmonics m = (m_0^0, m_1^-1, m_1^0, m_1^1, ..., m_N^N), index p = l^2 + l + k,
and the streaming matrices are A_d = int_{S^2} m m^T Omega_d dOmega.
Sec. 3.3.2: A_d = V_d Lambda_d V_d^T is split into A_d^+ = V_d max(Lambda_d, 0) V_d^T
and A_d^- = V_d min(Lambda_d, 0) V_d^T.

The real basis is written from its definition: for k > 0 it is
sqrt(2) N_lk P_l^k(mu) cos(k phi), for k = 0 it is N_l0 P_l(mu), for k < 0 it is
sqrt(2) N_l|k| P_l^|k|(mu) sin(|k| phi), with N_lk^2 = (2l+1)/(4 pi) (l-k)!/(l+k)!
and P_l^k the associated Legendre function WITHOUT the Condon-Shortley phase
(the paper's k > 0 formula reduces to this; its k < 0 formula is garbled and is
read as the matching sine function).

A_d is the definition evaluated by a product quadrature (Gauss-Legendre in mu,
uniform in phi) that is exact for the polynomial integrand.

Pins (tests/test_oracle_angular.py): quadrature orthonormality, the addition
theorem, eigenvalues of the k = 0 block of A_z equal to Gauss-Legendre nodes,
the textbook closed form of A_z, isospectrality of A_x, A_y, A_z.
"""
from __future__ import annotations

import numpy as np
from scipy.special import gammaln, lpmv


def n_moments(N: int) -> int:
    return (N + 1) ** 2


def moment_index(l: int, k: int) -> int:
    """p = l^2 + l + k (Sec. 3.3.1, moment vector ordering)."""
    return l * l + l + k


def degree_of_moment(N: int) -> np.ndarray:
    """l(p) for p = 0..m-1."""
    out = np.empty(n_moments(N), dtype=np.int64)
    for l in range(N + 1):
        for k in range(-l, l + 1):
            out[moment_index(l, k)] = l
    return out


def real_sh(N: int, mu: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """m(Omega) at directions (mu, phi); returns array (m, len(mu))."""
    mu = np.asarray(mu, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    out = np.zeros((n_moments(N), mu.size))
    for l in range(N + 1):
        for k in range(-l, l + 1):
            ka = abs(k)
            # scipy's lpmv carries the Condon-Shortley phase (-1)^k; remove it
            plk = lpmv(ka, l, mu) * (-1.0) ** ka
            norm = np.sqrt((2 * l + 1) / (4 * np.pi) * np.exp(gammaln(l - ka + 1) - gammaln(l + ka + 1)))
            if k == 0:
                val = norm * plk
            elif k > 0:
                val = np.sqrt(2.0) * norm * plk * np.cos(ka * phi)
            else:
                val = np.sqrt(2.0) * norm * plk * np.sin(ka * phi)
            out[moment_index(l, k)] = val
    return out


def real_sh_dir(N: int, omega) -> np.ndarray:
    """m(Omega) for one Cartesian unit direction (Omega_x, Omega_y, Omega_z)."""
    ox, oy, oz = (float(v) for v in omega)
    mu = np.clip(oz, -1.0, 1.0)
    phi = np.arctan2(oy, ox)
    return real_sh(N, np.array([mu]), np.array([phi]))[:, 0]


def sphere_quadrature(n_mu: int, n_phi: int):
    """Gauss-Legendre in mu times uniform (trapezoid) in phi.

    Exact for polynomials in Omega of degree <= min(2 n_mu - 1, n_phi - 1).
    Returns (mu, phi, weight) flattened.
    """
    x, wx = np.polynomial.legendre.leggauss(n_mu)
    phi = (np.arange(n_phi) + 0.5) * (2 * np.pi / n_phi)
    MU, PHI = np.meshgrid(x, phi, indexing="ij")
    W = np.outer(wx, np.full(n_phi, 2 * np.pi / n_phi))
    return MU.ravel(), PHI.ravel(), W.ravel()


def streaming_matrices(N: int):
    """A_x, A_y, A_z = int m m^T Omega_d dOmega (Sec. 3.3.1), exact quadrature."""
    n_mu = N + 2
    n_phi = 2 * N + 4
    mu, phi, w = sphere_quadrature(n_mu, n_phi)
    M = real_sh(N, mu, phi)  # (m, Q)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    om = (st * np.cos(phi), st * np.sin(phi), mu)
    A = []
    for d in range(3):
        Ad = (M * (w * om[d])) @ M.T
        Ad[np.abs(Ad) < 1e-14] = 0.0
        A.append(0.5 * (Ad + Ad.T))
    return A


def eigen_split(A: np.ndarray):
    """A^+ = V max(Lambda,0) V^T and A^- = V min(Lambda,0) V^T (Sec. 3.3.2)."""
    lam, V = np.linalg.eigh(A)
    Ap = (V * np.maximum(lam, 0.0)) @ V.T
    Am = (V * np.minimum(lam, 0.0)) @ V.T
    return Ap, Am, lam


class AngularTables:
    """Everything the method needs from the angular discretisation for degree N."""

    def __init__(self, N: int):
        self.N = N
        self.m = n_moments(N)
        self.A = streaming_matrices(N)
        self.Ap = []
        self.Am = []
        self.lam_max = []
        for d in range(3):
            ap, am, lam = eigen_split(self.A[d])
            self.Ap.append(ap)
            self.Am.append(am)
            self.lam_max.append(float(np.max(np.abs(lam))))
        self.degree = degree_of_moment(N)
