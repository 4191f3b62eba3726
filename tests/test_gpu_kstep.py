"""GPU parity of the streaming K-step (one energy step, RK4 sub-steps) through
the stand-alone C-ABI entry point dlra_kstep, against the oracle's K-step of
the augmented BUG streaming update (Sec. 2.2, Eq. KLS; Sec. 3.3.3)."""
import numpy as np
import pytest

from oracle import dlra as ODL
from oracle import problem as OP
from paper_2508_04484_gb300 import workloads as WL

from .gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def kstep_case(two_d, seed=3, r=6):
    if two_d:
        cfg = WL.base_config(nx=18, ny=1, nz=14, dx=0.2, dy=0.0, dz=0.2, N=3, collision=WL.BOLTZMANN,
                             e_max=80.0, e_min=20.0, n_steps=6, t100=2e-2)
    else:
        cfg = WL.base_config(nx=10, ny=9, nz=12, dx=0.2, dy=0.25, dz=0.2, N=3, collision=WL.BOLTZMANN,
                             e_max=80.0, e_min=20.0, n_steps=6, t100=2e-2)
    mats, w = WL.ellipsoid_phantom(cfg, seed, n_incl=3, semi=(0.3, 0.8))
    prob = OP.Problem(cfg, mats, w)
    rng = np.random.default_rng(seed)
    X, _ = np.linalg.qr(rng.standard_normal((prob.n, r)))
    W, _ = np.linalg.qr(rng.standard_normal((prob.m, r)))
    S = rng.standard_normal((r, r))
    k = 1
    Pk = []
    for d in prob.dirs:
        Pk.append(W.T @ prob.ang.Ap[d] @ W)
        Pk.append(W.T @ prob.ang.Am[d] @ W)
    rho_s = sum(prob.w[i] * m.density * m.sp_ratio for i, m in enumerate(prob.phys.mats))
    return cfg, prob, X, S, W, k, np.array(Pk), rho_s


def run_kstep(fn, cfg, prob, X, S, k, Pk, rho_s, K1=None):
    import torch
    from paper_2508_04484_gb300 import dlra as D
    dev = torch.device("cuda", 0)
    r = X.shape[1]
    K0 = torch.tensor(np.ascontiguousarray((X @ S).T), dtype=torch.float32, device=dev)
    if K1 is None:
        K1 = torch.zeros_like(K0)
    inv = torch.tensor(1.0 / rho_s, dtype=torch.float32, device=dev)
    P = torch.tensor(np.ascontiguousarray(np.transpose(Pk, (0, 2, 1))), dtype=torch.float32, device=dev)
    a = D.kstep_args(cfg, r, prob.E[k], prob.h, prob.n_sub(k), K0, K1, inv, P)
    fn(a)
    torch.cuda.synchronize()
    return K1.cpu().numpy().T.astype(np.float64)


@pytest.mark.parametrize("two_d", [True, False])
def test_kstep_matches_oracle(two_d):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    from paper_2508_04484_gb300 import dlra as D
    build.build()
    cfg, prob, X, S, W, k, Pk, rho_s = kstep_case(two_d)
    assert prob.n_sub(k) >= 2
    _, _, _, K1_ref, _ = ODL.streaming_bug(prob, X, S, W, k)
    K1 = run_kstep(D.dlra_kstep, cfg, prob, X, S, k, Pk, rho_s)
    assert rel_l2(K1, K1_ref) < 1e-5
