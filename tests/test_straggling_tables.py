"""The library's host tables of the straggling ray model (dlra_straggling_tables, C++) against
the oracle's energy-DG operators (oracle/straggling.py, NumPy): two independent assemblies of the
same discretisation (Sec. 3.2), compared entry by entry. Host only: no GPU needed."""
import numpy as np
import pytest

from oracle import straggling as ST


@pytest.fixture(scope="module")
def D():
    from paper_2508_04484_gb300 import build
    build.build()
    from paper_2508_04484_gb300 import dlra
    return dlra


def _dense(blocks):
    G = blocks.shape[0]
    M = np.zeros((3 * G, 3 * G))
    for e in range(G):
        for b in range(3):
            c = e - 1 + b
            if 0 <= c < G:
                M[3 * e:3 * e + 3, 3 * c:3 * c + 3] = blocks[e, b]
            else:
                assert np.all(blocks[e, b] == 0.0)
    return M


@pytest.mark.parametrize("straggling", [True, False])
@pytest.mark.parametrize("G,e_min,e_max", [(128, 1.0, 150.0), (16, 30.0, 66.0)])
def test_tables_match_the_oracle_operators(D, straggling, G, e_min, e_max):
    p, alpha, t100 = 1.77, 0.0022, 2e-2
    mass, adv, sipg, rem = D.straggling_tables(e_min, e_max, G, p, alpha, t100, straggling)
    dg = ST.EnergyDG(e_min, e_max, G)
    Sw = lambda E: E ** (1.0 - p) / (p * alpha)
    Tw = ST.straggling_water if straggling else (lambda E: 0.0 * np.asarray(E))
    rm = ST.RayMarch(dg, Sw, Tw, sigma_ref=lambda E: 0.5 * t100 * (100.0 / E) ** 2)
    assert np.allclose(mass, dg.mass, rtol=1e-15, atol=0.0)
    for lib, ora in ((adv, rm.B), (sipg, rm.K), (rem, rm.R)):
        L = _dense(lib)
        scale = np.abs(ora).max()
        # the oracle takes dT/dE by central differences: agreement to ~1e-9 of the largest entry
        assert np.abs(L - ora).max() <= 1e-9 * scale + 1e-300


def test_tables_reject_bad_arguments(D):
    with pytest.raises(D.DlraError):
        D.straggling_tables(10.0, 5.0, 16)
    with pytest.raises(D.DlraError):
        D.straggling_tables(0.0, 5.0, 16)


def test_a_march_on_the_library_tables_keeps_the_exact_moments(D):
    # constant-coefficient check through the library's blocks: with S and T constant the
    # Crank-Nicolson march conserves number and moves mean and variance exactly as the
    # continuous problem; here S = S_w(E) and T = T_w(E) vary, so check number conservation and
    # the exact energy balance of the slowing-down term instead
    e_min, e_max, G = 20.0, 120.0, 64
    mass, adv, sipg, rem = D.straggling_tables(e_min, e_max, G, 1.77, 0.0022, 0.0, True)
    dg = ST.EnergyDG(e_min, e_max, G)
    M = np.diag(mass)
    Gm = -_dense(adv) + _dense(sipg)
    h = 0.01
    A = M + 0.5 * h * Gm
    Bm = M - 0.5 * h * Gm
    c = dg.project(lambda E: np.exp(-0.5 * ((E - 100.0) / 1.5) ** 2))
    n0 = dg.number(c)
    for _ in range(300):
        c = np.linalg.solve(A, Bm @ c)
    assert abs(dg.number(c) / n0 - 1.0) < 1e-12
    m, v = dg.mean_var(c)
    assert m < 100.0 and v > 1.5 ** 2


def test_straggling_trace_rejects_bad_arguments_on_the_host(D):
    # argument checks run before any CUDA call
    import ctypes as C
    a = D.dlra_straggling_trace_args()
    a.nx = a.ny = a.nz = 4
    a.dx = a.dy = a.dz = 0.1
    a.e_min, a.e_max, a.n_bins, a.n_elem, a.h_max = 30.0, 60.0, 8, 16, 0.01
    a.bk_p, a.bk_alpha, a.t100, a.energy = 1.77, 0.0022, 1e-2, 70.0   # energy above e_max
    assert D.load().dlra_straggling_trace(C.byref(a)) == 1
    assert b"arguments" in D.load().dlra_last_error(None)
