"""Seeded synthetic inputs: grids, base materials, mixture phantoms and beams.

This module holds no arithmetic of the transport method. It only builds the
inputs both the CUDA library and the CPU oracle are given:

* configuration dictionaries (grid, angular degree, collision model, energy
  grid, rank control) shaped like the paper's test cases (Sec. 4: 1 mm and
  0.25 mm voxels, P_N expansions, truncation tolerance) and the five workloads
  used for measurement;
* base materials (water, cortical bone, lung) with a density, a stopping-power
  ratio, a scattering-power ratio and a screening parameter;
* mixture weights w_m(x) (Sec. 2.1, Eq. mixXS): seeded random ellipsoid
  inclusions of bone or lung in water, indicator fields smoothed by a Gaussian
  of one voxel and renormalised so that sum_m w_m(x) = 1;
* pencil beams (Sec. 4): Gaussian spot of 3 mm, energies, directions.
"""
from __future__ import annotations

import math

import numpy as np

FP, BOLTZMANN = 0, 1
FIXED, ADAPTIVE, SCHEDULE = 0, 1, 2
FP64, FP32_MIXED, FP32_SPLIT = 0, 1, 2

WATER = dict(density=1.0, sp_ratio=1.0, scatter_ratio=1.0, screening=1.0e-3)
BONE = dict(density=1.85, sp_ratio=0.90, scatter_ratio=1.35, screening=1.5e-3)
LUNG = dict(density=0.26, sp_ratio=1.0, scatter_ratio=1.0, screening=1.0e-3)


def base_config(**kw):
    cfg = dict(nx=8, ny=1, nz=8, dx=0.1, dy=0.0, dz=0.1, N=3, collision=BOLTZMANN,
               transport_correction=1, rank_mode=FIXED, rank=5, rank_max=64, trunc_tol=1e-3,
               e_max=100.0, e_min=1.0, n_steps=10, cfl=0.6, precision=FP64,
               bk_p=1.77, bk_alpha=0.0022, t100=1.72e-4)
    cfg.update(kw)
    return cfg


def homogeneous(cfg, material=WATER):
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return [dict(material)], np.ones((1, n))


def ellipsoid_phantom(cfg, seed, n_incl=12, semi=(0.5, 2.5), center_frac=0.6):
    """Water with seeded bone/lung ellipsoids; returns (materials, w (3, n))."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    dx, dy, dz = cfg["dx"], (cfg["dy"] if cfg["dy"] > 0 else 1.0), cfg["dz"]
    L = np.array([nx * dx, ny * dy, nz * dz])
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * dz, (np.arange(ny) + 0.5) * dy,
                          (np.arange(nx) + 0.5) * dx, indexing="ij")
    label = np.zeros((nz, ny, nx), dtype=np.int64)
    for _ in range(n_incl):
        c = L * (0.5 + center_frac * (rng.random(3) - 0.5))
        a = rng.uniform(semi[0], semi[1], size=3)
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        mat = 1 if rng.random() < 0.5 else 2
        d = np.stack([x - c[0], y - c[1], z - c[2]], axis=-1) @ q
        inside = np.sum((d / a) ** 2, axis=-1) <= 1.0
        label[inside] = mat
    w = np.zeros((3, nz, ny, nx))
    for m in range(3):
        ind = (label == m).astype(np.float64)
        w[m] = gaussian_filter(ind, sigma=1.0, mode="nearest")
    w /= w.sum(axis=0, keepdims=True)
    return [dict(WATER), dict(BONE), dict(LUNG)], w.reshape(3, -1)


def pencil_beam(energy, pos, direction=(0.0, 0.0, 1.0), spot_sigma=0.3, weight=1.0, energy_sigma=0.0):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return dict(energy=float(energy), energy_sigma=float(energy_sigma), pos=[float(v) for v in pos],
                dir=[float(v) for v in d], spot_sigma=float(spot_sigma), weight=float(weight))


def cone_beams(cfg, n_beams, seed, e_range=(70.0, 230.0), half_angle_deg=30.0, spot=0.3, face_frac=0.5):
    """Beams with energies U(e_range), directions uniform in a cone about +z, entry
    points uniform in the central face_frac of the z = 0 face."""
    rng = np.random.default_rng(seed)
    Lx, Ly = cfg["nx"] * cfg["dx"], cfg["ny"] * cfg["dy"]
    out = []
    cmin = math.cos(math.radians(half_angle_deg))
    for _ in range(n_beams):
        ct = rng.uniform(cmin, 1.0)
        st = math.sqrt(1 - ct * ct)
        ph = rng.uniform(0, 2 * math.pi)
        d = (st * math.cos(ph), st * math.sin(ph), ct)
        px = Lx * (0.5 + face_frac * (rng.random() - 0.5))
        py = Ly * (0.5 + face_frac * (rng.random() - 0.5))
        out.append(pencil_beam(rng.uniform(*e_range), (px, py, 0.0), d, spot))
    return out


# ---------------------------------------------------------------------------
# the five measured workloads (energies in MeV, lengths in cm)
# ---------------------------------------------------------------------------

def slab_fp_40x40():
    """2-D x-z slab 40x40 of 1 mm water, 100 MeV beam, Fokker-Planck, N=7, rank 5, 60 steps, FP64."""
    cfg = base_config(nx=40, ny=1, nz=40, dx=0.1, dy=0.0, dz=0.1, N=7, collision=FP,
                      transport_correction=0, rank_mode=FIXED, rank=5, rank_max=16,
                      e_max=100.0, e_min=1.0, n_steps=60, precision=FP64)
    mats, w = homogeneous(cfg)
    beams = [pencil_beam(100.0, (2.0, 0.0, 0.0))]
    return cfg, mats, w, beams


def water_64cube_boltzmann():
    """64^3 voxels of 2 mm water, 150 MeV, Boltzmann (eta=1e-3, ETC), N=15, rank 20, 200 steps."""
    cfg = base_config(nx=64, ny=64, nz=64, dx=0.2, dy=0.2, dz=0.2, N=15, collision=BOLTZMANN,
                      transport_correction=1, rank_mode=FIXED, rank=20, rank_max=20,
                      e_max=150.0, e_min=1.0, n_steps=200, precision=FP32_MIXED)
    mats, w = homogeneous(cfg)
    beams = [pencil_beam(150.0, (6.4, 6.4, 0.0))]
    return cfg, mats, w, beams


def phantom_128cube_adaptive(seed=3):
    """128^3 voxels of 1.5 mm, 3-material ellipsoid phantom, 180 MeV, N=21, adaptive tol 1e-3, r<=60."""
    cfg = base_config(nx=128, ny=128, nz=128, dx=0.15, dy=0.15, dz=0.15, N=21, collision=BOLTZMANN,
                      transport_correction=1, rank_mode=ADAPTIVE, rank=60, rank_max=60, trunc_tol=1e-3,
                      e_max=180.0, e_min=1.0, n_steps=358, precision=FP32_MIXED)
    mats, w = ellipsoid_phantom(cfg, seed)
    beams = [pencil_beam(180.0, (9.6, 9.6, 0.0))]
    return cfg, mats, w, beams


def phantom_96cube_32beams(seed=4):
    """96^3 voxels of 2 mm, phantom seed 4, 32 beams (70-230 MeV, 30 degree cone), N=21, ranks 10-40."""
    cfg = base_config(nx=96, ny=96, nz=96, dx=0.2, dy=0.2, dz=0.2, N=21, collision=BOLTZMANN,
                      transport_correction=1, rank_mode=ADAPTIVE, rank=40, rank_max=40, trunc_tol=1e-3,
                      e_max=230.0, e_min=1.0, n_steps=458, precision=FP32_MIXED)
    mats, w = ellipsoid_phantom(cfg, seed)
    beams = cone_beams(cfg, 32, seed)
    return cfg, mats, w, beams


def phantom_64cube_8beams(seed=5):
    """64^3 voxels of 2 mm, phantom seed 5, 8 beams with weights U(0.5, 1.5), 70-130 MeV."""
    cfg = base_config(nx=64, ny=64, nz=64, dx=0.2, dy=0.2, dz=0.2, N=15, collision=BOLTZMANN,
                      transport_correction=1, rank_mode=ADAPTIVE, rank=30, rank_max=30, trunc_tol=1e-3,
                      e_max=130.0, e_min=1.0, n_steps=258, precision=FP32_MIXED)
    mats, w = ellipsoid_phantom(cfg, seed)
    rng = np.random.default_rng(seed + 100)
    beams = cone_beams(cfg, 8, seed, e_range=(70.0, 130.0))
    for b in beams:
        b["weight"] = float(rng.uniform(0.5, 1.5))
    return cfg, mats, w, beams


def phantom_48cube_8beams(seed=6):
    """48^3 voxels of 2 mm, phantom seed 6, 8 beams (60-100 MeV, 30 degree cone), N=11,
    adaptive rank (tol 1e-3, <= 24), 120 energy steps: the batched-beam comparison case."""
    cfg = base_config(nx=48, ny=48, nz=48, dx=0.2, dy=0.2, dz=0.2, N=11, collision=BOLTZMANN,
                      transport_correction=1, rank_mode=ADAPTIVE, rank=24, rank_max=24, trunc_tol=1e-3,
                      e_max=100.0, e_min=1.0, n_steps=120, precision=FP32_MIXED)
    mats, w = ellipsoid_phantom(cfg, seed, n_incl=8, semi=(0.4, 1.8))
    beams = cone_beams(cfg, 8, seed, e_range=(60.0, 100.0))
    return cfg, mats, w, beams
