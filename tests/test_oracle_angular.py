"""Pins of the oracle's angular tables (Sec. 3.3.1, Sec. 3.3.2)."""
import numpy as np
import pytest

from oracle import angular as ang


@pytest.mark.parametrize("N", [1, 3, 7, 15])
def test_orthonormal_basis(N):
    mu, phi, w = ang.sphere_quadrature(N + 2, 2 * N + 4)
    M = ang.real_sh(N, mu, phi)
    assert np.abs((M * w) @ M.T - np.eye(ang.n_moments(N))).max() < 1e-12


@pytest.mark.parametrize("N", [3, 7])
def test_addition_theorem(N):
    # sum_p m_p(O) m_p(O') = sum_l (2l+1)/(4 pi) P_l(O . O') for any real orthonormal basis
    rng = np.random.default_rng(1)
    v = rng.standard_normal((2, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    a = ang.real_sh_dir(N, v[0])
    b = ang.real_sh_dir(N, v[1])
    c = np.array([(2 * l + 1) / (4 * np.pi) for l in range(N + 1)])
    ref = np.polynomial.legendre.legval(float(v[0] @ v[1]), c)
    assert abs(a @ b - ref) < 1e-12


@pytest.mark.parametrize("N", [3, 7, 15, 21])
def test_kzero_block_of_Az_has_gauss_nodes(N):
    T = ang.AngularTables(N)
    idx = [ang.moment_index(l, 0) for l in range(N + 1)]
    ev = np.sort(np.linalg.eigvalsh(T.A[2][np.ix_(idx, idx)]))
    gl = np.sort(np.polynomial.legendre.leggauss(N + 1)[0])
    assert np.abs(ev - gl).max() < 1e-12
    # lam_max of every A_d equals the largest Gauss-Legendre node of order N+1
    for d in range(3):
        assert abs(T.lam_max[d] - gl[-1]) < 1e-12


@pytest.mark.parametrize("N", [4, 7])
def test_Az_closed_form(N):
    # textbook: cos(theta) Y_l^k couples to Y_{l+1}^k with sqrt((l+1-k)(l+1+k)/((2l+1)(2l+3)))
    T = ang.AngularTables(N)
    Az = T.A[2]
    ref = np.zeros_like(Az)
    for l in range(N):
        for k in range(-l, l + 1):
            ka = abs(k)
            a = np.sqrt((l + 1 - ka) * (l + 1 + ka) / ((2 * l + 1) * (2 * l + 3)))
            p, q = ang.moment_index(l, k), ang.moment_index(l + 1, k)
            ref[p, q] = ref[q, p] = a
    assert np.abs(Az - ref).max() < 1e-13


@pytest.mark.parametrize("N", [3, 7])
def test_isospectral_symmetric_and_split(N):
    T = ang.AngularTables(N)
    ez = np.sort(np.linalg.eigvalsh(T.A[2]))
    for d in range(3):
        assert np.abs(T.A[d] - T.A[d].T).max() == 0.0
        assert np.abs(np.sort(np.linalg.eigvalsh(T.A[d])) - ez).max() < 1e-12
        assert np.abs(T.Ap[d] + T.Am[d] - T.A[d]).max() < 1e-12
        assert np.linalg.eigvalsh(T.Ap[d]).min() > -1e-12
        assert np.linalg.eigvalsh(T.Am[d]).max() < 1e-12


def test_streaming_moments_of_a_direction():
    # int m m^T Omega_d dOmega applied to m(O0): the l<=N-1 projection of Omega_d delta_{O0}
    # gives sum_d O0_d A_d m(O0) = m(O0)(O0 . O0) restricted to degrees < N  (plane-wave check)
    N = 6
    T = ang.AngularTables(N)
    v = np.array([0.3, -0.5, 0.81])
    v /= np.linalg.norm(v)
    m0 = ang.real_sh_dir(N, v)
    lhs = sum(v[d] * T.A[d] for d in range(3)) @ m0
    deg = ang.degree_of_moment(N)
    # exact identity for degrees <= N-1 (the projection of (Omega.v) m(v) is exact there)
    mask = deg <= N - 1
    # reference by quadrature of (Omega . v) sum_p m_p(Omega) m_p(v)
    mu, phi, w = ang.sphere_quadrature(N + 3, 2 * N + 6)
    M = ang.real_sh(N, mu, phi)
    st = np.sqrt(1 - mu * mu)
    od = st * np.cos(phi) * v[0] + st * np.sin(phi) * v[1] + mu * v[2]
    ref = (M * (w * od)) @ (M.T @ m0)
    assert np.abs(lhs[mask] - ref[mask]).max() < 1e-12
