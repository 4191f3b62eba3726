"""GPU parity of the stencil Gram G_k[a][b] = sum_i A(i, a) D_k(rho^-1 B(:, b))(i), the Galerkin
blocks of the streaming operator in the L-step and S-step (Sec. 3.3.2), through the stand-alone
C-ABI entry point dlra_stencil_gram: the FMA kernel, the tensor-core kernel (tcgen05 kind::tf32
with high/low splits) and the tensor-core kernel with a sliding TMA window (A == B, 3-D) against
the oracle's stencils (oracle/grid.py apply_D) in FP64 on the same FP32 inputs."""
import numpy as np
import pytest

from oracle import grid as OG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_04484_gb300 import build
    build.build()


def _oracle_gram(dims, spacing, A, B, inv_rho):
    two_d = dims[1] == 1 and spacing[1] == 0.0
    dirs = (0, 2) if two_d else (0, 1, 2)
    V = inv_rho[:, None] * B
    G = []
    for d in dirs:
        for sign in (-1, +1):
            G.append(OG.apply_D(V, dims, d, sign, spacing[d]).T @ A)
    return np.array(G)


def _case(dims, spacing, na, nb, seed, lda_pad=0):
    rng = np.random.default_rng(seed)
    n = dims[0] * dims[1] * dims[2]
    A = rng.standard_normal((na, n + lda_pad)).astype(np.float32)
    B = rng.standard_normal((nb, n + lda_pad)).astype(np.float32)
    inv_rho = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return A, B, inv_rho


def _gpu_gram(dims, spacing, A, B, inv_rho, variant):
    import torch
    from paper_2508_04484_gb300 import dlra as D
    dev = torch.device("cuda", 0)
    n = inv_rho.shape[0]
    # column-major n x na with leading dimension A.shape[1]: the transpose of a row-major (na, lda)
    At = torch.tensor(A, device=dev).T[:n]
    Bt = torch.tensor(B, device=dev).T[:n]
    r = torch.tensor(inv_rho, device=dev)
    G = D.stencil_gram(dims, spacing, At, Bt, r, variant=variant)
    torch.cuda.synchronize()
    return G.cpu().numpy()


# (grid, spacing, padding of the leading dimensions)
SHAPES = [
    ((13, 7, 9), (0.2, 0.25, 0.3), 3),   # 819 cells: 25 full 32-cell chunks and a ragged one
    ((37, 1, 21), (0.2, 0.0, 0.25), 3),  # x-z slab, nk = 4
    ((12, 5, 7), (0.2, 0.25, 0.3), 4),   # x-extent a multiple of 4 (float4 stencil loads), 420 cells
    ((20, 1, 9), (0.2, 0.0, 0.25), 8),   # the same on a slab, 180 cells
]


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("na,nb", [(20, 20), (40, 40), (7, 5), (64, 50), (128, 128), (16, 43)])
@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_stencil_gram_matches_oracle(shape, na, nb, variant):
    dims, spacing, pad = SHAPES[shape]
    A, B, inv_rho = _case(dims, spacing, na, nb, seed=10 + na + nb, lda_pad=pad)
    n = inv_rho.shape[0]
    Go = _oracle_gram(dims, spacing, A[:, :n].T.astype(np.float64), B[:, :n].T.astype(np.float64),
                      inv_rho.astype(np.float64))
    G = _gpu_gram(dims, spacing, A, B, inv_rho, variant)
    assert G.shape == Go.shape
    scale = np.abs(Go).max()
    # FP32 sums of a few hundred terms of size ~10: a few 1e-6 of the largest entry
    assert np.abs(G - Go).max() <= 3e-6 * scale
    for k in range(Go.shape[0]):
        assert np.linalg.norm(G[k] - Go[k]) <= 2e-6 * np.linalg.norm(Go[k])


@pytest.mark.parametrize("variant", [0, 1])
def test_stencil_gram_full_size_64cube(variant):
    # the shape of the augmented-basis Gram of the 64^3 workload: n2 = 40 columns on both sides
    dims, spacing = (64, 64, 64), (0.2, 0.2, 0.2)
    A, B, inv_rho = _case(dims, spacing, 40, 40, seed=5)
    Go = _oracle_gram(dims, spacing, A.T.astype(np.float64), B.T.astype(np.float64), inv_rho.astype(np.float64))
    G = _gpu_gram(dims, spacing, A, B, inv_rho, variant)
    # 262144-term sums: FP32 within a block, FP64 across blocks
    for k in range(Go.shape[0]):
        assert np.linalg.norm(G[k] - Go[k]) <= 2e-5 * np.linalg.norm(Go[k])


def test_stencil_gram_same_basis_is_the_solver_shape():
    # A = B (the L-step and S-step case): both kernels agree to FP32 round-off
    dims, spacing = (16, 16, 16), (0.25, 0.25, 0.25)
    A, _, inv_rho = _case(dims, spacing, 24, 1, seed=8)
    G0 = _gpu_gram(dims, spacing, A, A, inv_rho, 0)
    G1 = _gpu_gram(dims, spacing, A, A, inv_rho, 1)
    assert np.linalg.norm(G1 - G0) <= 2e-6 * np.linalg.norm(G0)


def test_stencil_gram_rejects_bad_arguments():
    import torch
    from paper_2508_04484_gb300 import dlra as D
    dev = torch.device("cuda", 0)
    X = torch.zeros((129, 64), dtype=torch.float32, device=dev).T   # 64 cells x 129 columns
    r = torch.ones(64, dtype=torch.float32, device=dev)
    with pytest.raises(D.DlraError):
        D.stencil_gram((4, 4, 4), (0.1, 0.1, 0.1), X, X, r)


def _kernel_names(fn):
    # names of the CUDA kernels fn launches (empty where the profiler records none)
    import torch
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    return {e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA}


# 3-D grids with nx % 4 == 0: one ragged run (nx < 32), whole and ragged runs, short lines
WIN_SHAPES = [
    ((12, 5, 7), (0.2, 0.25, 0.3), 4),
    ((20, 18, 10), (0.2, 0.2, 0.2), 0),
    ((36, 7, 5), (0.25, 0.2, 0.3), 8),
    ((64, 9, 11), (0.2, 0.3, 0.25), 0),
]


@pytest.mark.parametrize("nb", [20, 40, 64, 100, 128])
@pytest.mark.parametrize("shape", range(len(WIN_SHAPES)))
def test_windowed_stencil_gram_matches_oracle(shape, nb):
    # A == B (one device array, as in the L-step and S-step): 64-column and 128-column forms
    import torch
    from paper_2508_04484_gb300 import dlra as D
    dims, spacing, pad = WIN_SHAPES[shape]
    A, _, inv_rho = _case(dims, spacing, nb, 1, seed=30 + nb + shape, lda_pad=pad)
    n = inv_rho.shape[0]
    Go = _oracle_gram(dims, spacing, A[:, :n].T.astype(np.float64), A[:, :n].T.astype(np.float64),
                      inv_rho.astype(np.float64))
    dev = torch.device("cuda", 0)
    At = torch.tensor(A, device=dev).T[:n]
    r = torch.tensor(inv_rho, device=dev)
    out = {}

    def run():
        out["G"] = D.stencil_gram(dims, spacing, At, At, r, variant=2)

    names = _kernel_names(run)
    if names:
        assert any("gram_win_kernel" in k for k in names), sorted(names)
    G = out["G"].cpu().numpy()
    # each tensor-core sum runs over at most 8 chunks x 12 MMAs = 96 roundings toward zero:
    # a same-sign sum (the diagonal) may lose up to 96 x 2^-24 = 5.7e-6 of itself
    scale = np.abs(Go).max()
    assert np.abs(G - Go).max() <= 6e-6 * scale
    for k in range(Go.shape[0]):
        assert np.linalg.norm(G[k] - Go[k]) <= 6e-6 * np.linalg.norm(Go[k])


@pytest.mark.parametrize("nb", [64, 128])
def test_windowed_stencil_gram_full_size_64cube(nb):
    # 262,144 cells, the r x r and 2r x 2r widths of the solver's Grams, A == B: the three
    # kernels against the oracle. The first tensor-core kernel keeps a block's partial sums in
    # FP32 in tensor memory over ~3,500 cells, i.e. ~1,300 MMA roundings per entry; the tensor
    # core's FP32 accumulation rounds toward zero, so a same-sign sum (the diagonal, dominated by
    # the -3 v0 term of the one-sided stencils on random data) shrinks by up to that many units
    # in the last place: expected ~N 2^-25 = 4e-5, at most N 2^-23 = 1.6e-4 (bound 2.3e-4). The
    # windowed kernel restarts its tensor-core sums every 8 chunks (96 roundings, < 1.2e-5) and
    # adds them with round-to-nearest FP32 additions
    import torch
    from paper_2508_04484_gb300 import dlra as D
    dims, spacing = (64, 64, 64), (0.2, 0.2, 0.2)
    A, _, inv_rho = _case(dims, spacing, nb, 1, seed=7 + nb)
    Go = _oracle_gram(dims, spacing, A.T.astype(np.float64), A.T.astype(np.float64), inv_rho.astype(np.float64))
    dev = torch.device("cuda", 0)
    At = torch.tensor(A, device=dev).T
    r = torch.tensor(inv_rho, device=dev)
    G = {v: D.stencil_gram(dims, spacing, At, At, r, variant=v).cpu().numpy() for v in (0, 1, 2)}
    err = {v: max(np.linalg.norm(G[v][k] - Go[k]) / np.linalg.norm(Go[k]) for k in range(Go.shape[0]))
           for v in G}
    print(f"64^3, {nb} columns, A == B: relative error of the FMA / tensor-core / windowed Grams "
          f"{err[0]:.2e} / {err[1]:.2e} / {err[2]:.2e}")
    assert err[0] <= 2e-5
    assert err[1] <= 2.3e-4
    assert err[2] <= 1.2e-5
