"""GPU parity at the full 128^3 size of the timed workload (1.5 mm voxels, the three-material
phantom of seed 3), in the launch configurations the bench times, on sampled outputs that the
oracle computes one by one.

* The streaming K-step with the tensor-core stage the autotuner keeps (kernel 13: five TMA boxes
  per chunk, eight formation warps, A operand in TMEM) and the one it kept before (kernel 7) at
  rank 60 (capacity 64), one RK4 sub-step (an energy step of 0.03 MeV): every output cell
  depends on the input within eight cells (four stages of a two-cell stencil), so the oracle's
  K-step (Sec. 2.2 Eq. KLS, Sec. 3.3.2-3.3.3) on the 17^3 box around a sampled cell, with the
  same materials, gives that cell's K1 row exactly; cells on faces, edges and corners of the
  grid keep their vacuum ghost layer.
* The windowed stencil Gram (kernel 2) at the solver's two widths, 64 and 128 columns: sampled
  entries G_k[a][b] = sum_i X(i, a) D_k(rho^-1 X(:, b))(i) in FP64 from the oracle's stencils.

The locality the K-step check rests on is itself checked on the CPU: the oracle on a radius-8
box reproduces its full-grid row exactly, and on a radius-7 box it does not.
"""
import numpy as np
import pytest

from oracle import problem as OP
from oracle.fullrank import rk4
from oracle.grid import apply_D
from paper_2508_04484_gb300 import workloads as WL

DIMS = (128, 128, 128)
SPACING = (0.15, 0.15, 0.15)
# sampled cells (x, y, z): interior, faces, an edge and a corner
CELLS = [(64, 64, 64), (0, 70, 33), (127, 5, 90), (40, 0, 127), (1, 126, 1), (127, 127, 0), (90, 31, 2)]


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    build.build()


def _cell(x, y, z, dims):
    return (z * dims[1] + y) * dims[0] + x


def _kstep_config(dims):
    return WL.base_config(nx=dims[0], ny=dims[1], nz=dims[2], dx=SPACING[0], dy=SPACING[1], dz=SPACING[2], N=7,
                          collision=WL.BOLTZMANN, e_max=180.0, e_min=179.97, n_steps=1)


def _fK(prob, Pp, Pm):
    """Right-hand side of the K equation (Sec. 2.2) as the oracle's BUG step writes it."""
    def fK(t, K):
        Y = K / prob.stopping(prob.energy_at(t))[:, None]
        out = np.zeros_like(K)
        for d in prob.dirs:
            out += apply_D(Y, prob.dims, d, -1, prob.delta[d]) @ Pp[d]
            out += apply_D(Y, prob.dims, d, +1, prob.delta[d]) @ Pm[d]
        return out
    return fK


def _subbox_k1(cfg, mats, w, dims, K0h, Pp, Pm, c, R=8):
    """K1 row of cell c after one RK4 step of the oracle on the box of radius R around c
    (clipped to the grid, whose faces keep their zero ghost layers)."""
    lo = [max(v - R, 0) for v in c]
    hi = [min(v + R, n - 1) for v, n in zip(c, dims)]
    sub = tuple(h - l + 1 for l, h in zip(lo, hi))
    zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                             np.arange(lo[0], hi[0] + 1), indexing="ij")
    idx = ((zz * dims[1] + yy) * dims[0] + xx).reshape(-1)
    ps = OP.Problem(dict(cfg, nx=sub[0], ny=sub[1], nz=sub[2]), mats, w[:, idx])
    assert ps.n_sub(0) == 1
    K1s = rk4(_fK(ps, Pp, Pm), 0.0, K0h[:, idx].T.astype(np.float64), ps.h, 1)
    return K1s[_cell(c[0] - lo[0], c[1] - lo[1], c[2] - lo[2], sub)]


def _projections(prob, r, rng):
    W, _ = np.linalg.qr(rng.standard_normal((prob.m, r)))
    Pp = {d: W.T @ prob.ang.Ap[d] @ W for d in prob.dirs}
    Pm = {d: W.T @ prob.ang.Am[d] @ W for d in prob.dirs}
    return Pp, Pm


def test_subbox_kstep_equals_full_grid():
    """One RK4 step reaches eight cells (four stages of a two-cell stencil), so the oracle on
    the radius-8 box around a cell gives the full grid's row there exactly; on radius 7 an
    interior cell's row changes."""
    dims = (30, 28, 26)
    cfg = _kstep_config(dims)
    mats, w = WL.ellipsoid_phantom(cfg, 3)
    prob = OP.Problem(cfg, mats, w)
    assert prob.n_sub(0) == 1
    rng = np.random.default_rng(11)
    Pp, Pm = _projections(prob, 12, rng)
    K0h = rng.standard_normal((12, prob.n), dtype=np.float32)
    full = rk4(_fK(prob, Pp, Pm), 0.0, K0h.T.astype(np.float64), prob.h, 1)
    for c in [(15, 14, 13), (0, 3, 25), (29, 27, 0), (9, 0, 12)]:
        got = _subbox_k1(cfg, mats, w, dims, K0h, Pp, Pm, c)
        assert np.array_equal(got, full[_cell(*c, dims)]), c
    c = (15, 14, 13)
    assert not np.allclose(_subbox_k1(cfg, mats, w, dims, K0h, Pp, Pm, c, R=7), full[_cell(*c, dims)],
                           rtol=1e-12, atol=0.0)


@pytest.mark.gpu
@pytest.mark.parametrize("stage_kernel", [7, 13])
def test_kstep_tensor_core_stage_full_size_sampled(built, stage_kernel):
    import torch
    from paper_2508_04484_gb300 import dlra as D
    cfg = _kstep_config(DIMS)
    mats, w = WL.ellipsoid_phantom(cfg, 3)
    prob = OP.Problem(cfg, mats, w)
    assert prob.n_sub(0) == 1
    r = 60
    rng = np.random.default_rng(11)
    Pp, Pm = _projections(prob, r, rng)
    Pk = []
    for d in prob.dirs:
        Pk += [Pp[d], Pm[d]]
    rho_s = sum(prob.w[i] * m.density * m.sp_ratio for i, m in enumerate(prob.phys.mats))
    K0h = rng.standard_normal((r, prob.n), dtype=np.float32)   # column-major n x r
    dev = torch.device("cuda", 0)
    K0 = torch.tensor(K0h, device=dev)
    K1 = torch.zeros_like(K0)
    inv = torch.tensor(1.0 / rho_s, dtype=torch.float32, device=dev)
    P = torch.tensor(np.ascontiguousarray(np.transpose(np.array(Pk), (0, 2, 1))), dtype=torch.float32, device=dev)
    a = D.kstep_args(cfg, r, prob.E[0], prob.h, 1, K0, K1, inv, P, stage_kernel=stage_kernel)
    D.dlra_kstep(a)
    torch.cuda.synchronize()
    K1h = K1.cpu().numpy()
    worst = 0.0
    for c in CELLS:
        ref = _subbox_k1(cfg, mats, w, DIMS, K0h, Pp, Pm, c)
        got = K1h[:, _cell(*c, DIMS)].astype(np.float64)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        worst = max(worst, err)
        assert err < 1e-5, (c, err)
    print(f"K-step at 128^3, rank 60, stage kernel {stage_kernel}: worst sampled-row error {worst:.2e} over "
          f"{len(CELLS)} cells")


@pytest.mark.gpu
@pytest.mark.parametrize("nb", [64, 128])
def test_windowed_stencil_gram_full_size_sampled(built, nb):
    import torch
    from paper_2508_04484_gb300 import dlra as D
    cfg = _kstep_config(DIMS)
    mats, w = WL.ellipsoid_phantom(cfg, 3)
    rho = sum(w[i] * m["density"] * m["sp_ratio"] for i, m in enumerate(mats))
    n = int(np.prod(DIMS))
    rng = np.random.default_rng(40 + nb)
    Ah = rng.standard_normal((nb, n), dtype=np.float32)
    dev = torch.device("cuda", 0)
    A = torch.tensor(Ah, device=dev).T
    inv = torch.tensor(1.0 / rho, dtype=torch.float32, device=dev)
    G = D.stencil_gram(DIMS, SPACING, A, A, inv, variant=2).cpu().numpy()   # (nk, nb, na)
    inv64 = (1.0 / rho).astype(np.float32).astype(np.float64)
    picks = [(0, 3, 3), (1, 7, 7), (2, 0, 5), (3, nb - 1, nb - 1), (4, 10, nb // 2), (5, nb // 2, 1)]
    worst = 0.0
    for (kk, b, aa) in picks:
        d, sign = kk // 2, (-1 if kk % 2 == 0 else +1)
        vb = (inv64 * Ah[b].astype(np.float64))[:, None]
        ref = float(apply_D(vb, DIMS, d, sign, SPACING[d])[:, 0] @ Ah[aa].astype(np.float64))
        # the scale of a same-sign sum of the same terms: the bound of the restarted tensor-core sums
        scale = float(np.abs(apply_D(vb, DIMS, d, sign, SPACING[d])[:, 0] * Ah[aa]).sum())
        err = abs(float(G[kk, b, aa]) - ref) / scale
        worst = max(worst, err)
        assert err < 6e-6, (kk, b, aa, G[kk, b, aa], ref, scale)
    print(f"windowed stencil Gram at 128^3 x {nb}: worst sampled error {worst:.2e} of the entry's absolute sum")
