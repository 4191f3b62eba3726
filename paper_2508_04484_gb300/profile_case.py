"""Small profiling cases for single-kernel captures (ncu) of the heavy kernels.

A full capture replays a kernel about forty times and saves and restores the device memory
between replays, so it is run on a case a few GB in size whose buffers still exceed L2:

  python -m paper_2508_04484_gb300.profile_case stage --variant 4
      one energy step of a 96^3 three-material phantom (1.5 mm, P_21, rank 60 state, the
      128^3 workload's voxels, physics and rank capacity) with a chosen streaming-stage
      kernel (0 per-cell FMA, 3 cell pairs, 4 .. 13 the tensor-core forms of
      Solver.set_stage_kernel, 13 the five-box form the autotuner keeps);
  python -m paper_2508_04484_gb300.profile_case gram --variant 2
      the same step with a chosen stencil-Gram kernel (0 FMA, 1 tensor cores, 2 tensor cores
      with the sliding TMA window); the step launches it twice (r x r and 2r x 2r);
  --gram-kernel 1 runs the step's tall-skinny Grams on the tensor cores (gram_tt_kernel).

Seeded synthetic inputs (workloads.ellipsoid_phantom, random orthonormal factors with
decaying singular values); prints the rank log of the step.
"""
from __future__ import annotations

import argparse

import numpy as np


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["stage", "gram"])
    p.add_argument("--variant", type=int, default=4)
    p.add_argument("--edge", type=int, default=96)
    p.add_argument("--gram-kernel", type=int, default=0, help="tall-skinny Grams: 0 FMA, 1 tensor cores")
    a = p.parse_args(argv)
    import torch

    from . import build as B
    from . import dlra as D
    from . import workloads as WL

    B.build()
    e = a.edge
    cfg = WL.base_config(nx=e, ny=e, nz=e, dx=0.15, dy=0.15, dz=0.15, N=21, collision=WL.BOLTZMANN,
                         transport_correction=1, rank_mode=WL.FIXED, rank=60, rank_max=60, e_max=180.0,
                         e_min=178.0, n_steps=4, precision=WL.FP32_MIXED)
    mats, w = WL.ellipsoid_phantom(cfg, 3)
    beams = [WL.pencil_beam(180.0, (0.075 * e, 0.075 * e, 0.0), spot_sigma=0.3)]
    torch.cuda.set_device(0)
    s = D.Solver(cfg, mats, w, beams)
    n = e ** 3
    m = (cfg["N"] + 1) ** 2
    r = 60
    rng = np.random.default_rng(0)
    X = np.linalg.qr(rng.standard_normal((n, r)))[0]
    W = np.linalg.qr(rng.standard_normal((m, r)))[0]
    S = np.diag(1e-2 * 0.9 ** np.arange(r))
    s.set_state(X, S, W)
    if a.case == "stage":
        s.set_stage_kernel(a.variant)
        s.set_stencil_gram_kernel(1)
    else:
        s.set_stage_kernel(4)
        s.set_stencil_gram_kernel(a.variant)
    s.set_gram_kernel(a.gram_kernel)
    s.step(1)
    torch.cuda.synchronize()
    print("rank log of the step:", s.rank_log()[0].tolist())
    s.close()


if __name__ == "__main__":
    main()
