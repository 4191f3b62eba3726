"""GPU parity of the straggling ray trace (dlra_straggling_trace, Sec. 3.2) against the oracle's
energy-DG tracer (oracle/straggling.py trace_straggling): the same discretisation (128 P2 energy
elements, Lax-Friedrichs slowing down, SIPG straggling, Crank-Nicolson steps <= 0.01 cm), so the
bin-averaged fluence and the deposit agree to FP64 round-off. A host build of the same
preparation and per-ray march matches the oracle to 3e-15 on these cases
(tests/test_straggling_host_march.py)."""
import numpy as np
import pytest

from oracle import problem as OP
from oracle import straggling as ST
from paper_2508_04484_gb300 import workloads as WL

from .gpu_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    build.build()


def _factors(cfg, mats, w):
    prob = OP.Problem(cfg, mats, w)
    f = np.zeros(prob.n)
    for i, m in enumerate(prob.phys.mats):
        f += prob.w[i] * m.density * m.sp_ratio
    E = 50.0
    tau = sum(prob.w[i] * prob.phys.sigma_t(i, E) for i in range(prob.M)) / (0.5 * cfg["t100"] * (100.0 / E) ** 2)
    return prob, f, np.asarray(tau, dtype=np.float64)


CASES = [
    ("slab", dict(spot_sigma=0.0, energy_sigma=0.0), False),
    ("slab", dict(spot_sigma=0.1, energy_sigma=1.5), True),
    ("cube", dict(spot_sigma=0.15, energy_sigma=1.0), True),
]


@pytest.mark.parametrize("case,beam_kw,straggling", CASES)
def test_straggling_trace_matches_oracle(case, beam_kw, straggling):
    import torch
    from paper_2508_04484_gb300 import dlra as D
    if case == "slab":
        cfg = WL.base_config(nx=16, ny=1, nz=20, dx=0.2, dy=0.0, dz=0.2, N=3, collision=WL.BOLTZMANN,
                             e_max=66.0, e_min=30.0, n_steps=8, precision=WL.FP64, t100=2e-2)
        mats, w = WL.homogeneous(cfg)
        beam = WL.pencil_beam(60.0, (1.3, 0.0, 0.0), (0.2, 0.0, 1.0), **beam_kw)
        G = 128
    else:
        cfg = WL.base_config(nx=8, ny=7, nz=10, dx=0.25, dy=0.25, dz=0.25, N=3, collision=WL.BOLTZMANN,
                             e_max=62.0, e_min=30.0, n_steps=6, precision=WL.FP64, t100=2e-2)
        mats, w = WL.ellipsoid_phantom(cfg, 5, n_incl=3, semi=(0.3, 0.8))
        beam = WL.pencil_beam(58.0, (1.0, 0.9, 0.0), (0.15, -0.1, 1.0), **beam_kw)
        G = 64
    prob, f, tau = _factors(cfg, mats, w)
    dev = torch.device("cuda", 0)
    psi, e_u = D.straggling_trace(cfg, beam, torch.tensor(f, device=dev), torch.tensor(tau, device=dev),
                                  n_elem=G, straggling=straggling)
    ref = ST.trace_straggling(prob, beam, n_elem=G, h_max=0.01, straggling=straggling)
    assert rel_l2(e_u.cpu().numpy(), ref.e_u) < 1e-12
    assert rel_l2(psi.cpu().numpy(), ref.psi) < 1e-12


@pytest.mark.parametrize("straggling", [False, True])
def test_solver_with_straggling_source_matches_oracle(straggling):
    # the solver's uncollided source from the energy-DG tracer (dlra_set_straggling) against the
    # oracle's low-rank solve driven by its own energy-DG tracer (oracle/straggling.py)
    from oracle import dlra as ODL
    from paper_2508_04484_gb300 import dlra as D
    cfg = WL.base_config(nx=16, ny=1, nz=20, dx=0.2, dy=0.0, dz=0.2, N=3, collision=WL.BOLTZMANN,
                         rank_mode=WL.FIXED, rank=4, rank_max=8, e_max=66.0, e_min=30.0, n_steps=8,
                         precision=WL.FP64, t100=2e-2)
    mats, w = WL.homogeneous(cfg)
    beam = WL.pencil_beam(60.0, (1.3, 0.0, 0.0), (0.2, 0.0, 1.0), spot_sigma=0.1, energy_sigma=1.5)
    prob = OP.Problem(cfg, mats, w)
    tr = ST.trace_straggling(prob, beam, n_elem=128, h_max=0.01, straggling=straggling)
    d = np.asarray(beam["dir"]) / np.linalg.norm(beam["dir"])
    ref = ODL.solve(prob, [(tr.psi, tr.e_u, d)], ODL.RankControl(mode=OP.FIXED, rank=4))
    c = dict(cfg, rank_mode=WL.SCHEDULE, rank_schedule=ref["ranks"])
    s = D.Solver(c, mats, w, [beam])
    s.set_straggling(True, n_elem=128, h_max=0.01, straggling=straggling)
    psi0, e_u = s.source(2)
    assert rel_l2(psi0, tr.psi[2]) < 1e-12
    assert rel_l2(e_u, tr.e_u) < 1e-12
    dose = s.run()
    assert np.array_equal(s.rank_log(), ref["ranks"])
    err = rel_l2(dose, ref["dose"])
    print(f"solver with the energy-DG source (straggling {straggling}): dose error {err:.2e}")
    assert err < 1e-9
    s.close()
