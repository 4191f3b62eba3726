"""Throughput of the low-rank collided-proton transport solve on GB300.

Headline workload: the 128^3 heterogeneous phantom (1.5 mm voxels, three base materials by the
mixture model: water, cortical bone, lung; seeded ellipsoid inclusions), one 180 MeV pencil beam,
Boltzmann screened-Rutherford scattering with the extended transport correction, P_21 (484
moments), adaptive rank (truncation tolerance 1e-3 relative, at most 60), 358 energy steps
180 -> 1 MeV, FP32 streaming stage and contractions with FP64 orthonormalisation (pivoted
CholeskyQR2 factors on the cell side, Householder QR and Gram-Schmidt on the moment side).

A bench step is a run of consecutive energy steps of the solve: with K timed steps each runs
ceil(358 / K) energy steps, so the K timed steps together are one whole solve (the ray trace at
the start of the first step, every energy step with its streaming BUG step, collided scattering,
first-collision source and truncations, the dose read at the end of the last step). value =
energy steps / s over the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores, each step one energy step of a
bounded sample of the same workload (a 12^3 block of the phantom), scaled to the whole grid.
Under torchrun each rank solves its own copy of the single-beam workload (weak scaling); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "energy steps/s and cell·rank updates/s per GB300, % HBM roofline, vs plain"
UNIT = "energy steps/s"
WORKLOAD = "phantom_128cube_adaptive"
SECOND = "water_64cube_boltzmann"
WORKLOADS = [WORKLOAD, SECOND, "phantom_48cube_8beams", "phantom_96cube_32beams", "phantom_64cube_8beams",
             "slab_fp_40x40"]
PRECISION_NAMES = {0: "FP64", 1: "FP32-mixed (FP32 stage, contractions, SVD and S-step; FP64 orthonormalisation)",
                   2: "FP32-split (FP32 stage and contractions; FP64 orthonormalisation, truncation SVD and S-step)"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD, choices=WORKLOADS)
    p.add_argument("--precision", type=int, choices=[0, 1, 2], default=None,
                   help="override the workload's precision (0 FP64, 1 FP32-mixed, 2 FP32-split)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-second", action="store_true", help="skip the 64^3 water line")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched-against-plain comparison on the 64^3 eight-beam phantom")
    p.add_argument("--no-adjoint", action="store_true", help="skip timing the reverse sweep (dlra_backward)")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch variants")
    p.add_argument("--stage-kernel", type=int, choices=list(range(14)), default=None,
                   help="profiling: streaming-stage kernel (0 per-cell FMA, 1 tensor cores, 2 brick, 3 cell pairs, "
                        "4 / 5 TMA-staged tensor cores, 128 / 256-cell bricks, 6 persistent, 7 A in TMEM, "
                        "8 2-CTA clusters, 9 three tiles along z, 10 eight-column chunks, 11 eight formation warps, 12 five boxes and an FP32 B image, "
                        "13 five boxes and the split B image), "
                        "set after the autotuner")
    p.add_argument("--stencil-gram-kernel", type=int, choices=[0, 1, 2], default=None,
                   help="profiling: stencil-Gram kernel (0 FMA, 1 tensor cores, 2 tensor cores with a TMA window), "
                        "set after the autotuner")
    p.add_argument("--gram-kernel", type=int, choices=[0, 1], default=None,
                   help="profiling: tall-skinny Grams (0 FMA, 1 tensor cores), set after the autotuner")
    p.add_argument("--apply-kernel", type=int, choices=[0, 1, 2], default=None,
                   help="profiling: tall-skinny products (0 FMA, 1 tensor cores from 65,536 rows, 2 always), "
                        "set after the autotuner")
    p.add_argument("--replicas", action="store_true",
                   help="with several ranks, solve the whole multi-beam workload on every rank")
    p.add_argument("--graphs", default="auto", choices=["auto", "on", "off"],
                   help="replay the energy steps from CUDA graphs (auto: on for multi-beam workloads)")
    p.add_argument("--energy-steps", type=int, default=0,
                   help="profiling only: stop each solve after this many energy steps")
    return p.parse_args()


def _workload(name=WORKLOAD):
    from paper_2508_04484_gb300 import workloads as WL
    return getattr(WL, name)()


# streaming-stage kernels by variant: name and the markers of their source text (device.cuh
# unless a file is given; the DRAM traffic of a capture is reported only while that text is
# unchanged)
STAGE_KERNELS = {
    0: ("kstage_kernel", "template <typename T, int RM, int NACT>\n__global__ void __launch_bounds__(128) kstage_kernel(",
        "// The streaming stage of kstage_kernel on the FP32 path with two"),
    1: ("kstage_tc_kernel", None, None),
    2: ("kstage_brick_kernel", "// Cell bricks of the staged streaming stage", None),
    3: ("kstage_pair_kernel", "// The streaming stage of kstage_kernel on the FP32 path with two",
        "// Cell bricks of the staged streaming stage"),
    4: ("kstage_tma_kernel", None, None),
    5: ("kstage_tma_kernel", None, None),
    6: ("kstage_tmap_kernel", None, None),
    7: ("kstage_tmaa_kernel", "template <int RM>\n__global__ void __launch_bounds__(192) kstage_tmaa_kernel(",
        "}  // namespace dlra", "kstage_tma.cuh"),
    8: ("kstage_tmac_kernel", "template <int RM>\n__global__ void __launch_bounds__(192) kstage_tmac_kernel(",
        "}  // namespace dlra", "kstage_tmac.cuh"),
    9: ("kstage_tmat_kernel", "template <int RM, int T>\n__global__ void __launch_bounds__(KsTmaT<RM, T>::THREADS, 1)",
        "}  // namespace dlra", "kstage_tmat.cuh"),
    10: ("kstage_tmaa8_kernel", "template <int RM>\n__global__ void __launch_bounds__(192) kstage_tmaa8_kernel(",
         "}  // namespace dlra", "kstage_tma8.cuh"),
    11: ("kstage_tmaw_kernel", "template <int RM>\n__global__ void __launch_bounds__(320, 2) kstage_tmaw_kernel(",
         "}  // namespace dlra", "kstage_tmaw.cuh"),
    12: ("kstage_tmaf_kernel", "template <int RM, bool SPLIT>\n__global__ void __launch_bounds__(320, 2) kstage_tmaf_kernel(",
         "}  // namespace dlra", "kstage_tmaf.cuh"),
    13: ("kstage_tmaf_kernel", "template <int RM, bool SPLIT>\n__global__ void __launch_bounds__(320, 2) kstage_tmaf_kernel(",
         "}  // namespace dlra", "kstage_tmaf.cuh"),
}
STAGE_NAMES = {"per-cell FMA": 0, "tensor cores": 1, "brick FMA": 2, "cell pairs": 3, "TMA tensor cores 128": 4,
               "TMA tensor cores 256": 5, "TMA tensor cores persistent": 6, "TMA tensor cores A in TMEM": 7,
               "TMA tensor cores cluster": 8,
               "TMA tensor cores 3 tiles": 9,
               "TMA tensor cores 8 columns": 10, "TMA tensor cores 8 formation warps": 11,
               "TMA tensor cores faces": 12, "TMA tensor cores faces split B": 13}
GRAM_NAMES = {"FMA": 0, "tensor cores": 1, "tensor cores TMA window": 2}
APPLY_NAMES = {"FMA": 0, "tensor cores": 1}


def stage_source_sha256(variant):
    """sha256 of the source text of a streaming-stage kernel, or None without markers."""
    import hashlib
    rec = STAGE_KERNELS[variant]
    begin, end = rec[1], rec[2]
    fname = rec[3] if len(rec) > 3 else "device.cuh"
    if begin is None or end is None:
        return None
    src = open(os.path.join(ROOT, "paper_2508_04484_gb300", "csrc", fname)).read()
    i = src.find(begin)
    j = src.find(end, i + 1) if i >= 0 else -1
    if i < 0 or j < i:
        return None
    return hashlib.sha256(src[i:j].encode()).hexdigest()


def _stage_traffic(variant, workload=WORKLOAD, n=None, mean_words=None):
    """DRAM bytes per launch of the streaming-stage kernel in use on this workload from the
    committed ncu summary, or None when there is none or the kernel's source changed since.
    A capture of a smaller case of the workload records its bytes per cell and (5r + 1) word;
    they are scaled to n cells and the solve's mean (5r + 1) words per cell and launch."""
    name = STAGE_KERNELS[variant][0]
    path = os.path.join(ROOT, "profiles", "kstage_traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f).get("workloads", {}).get(workload, {}).get("kernels", {}).get(name)
    if d is None:
        return None, f"no capture of {name} on {workload}"
    h = stage_source_sha256(variant)
    if h is None or d.get("source_sha256") != h:
        return None, "kernel changed since the capture"
    if "dram_bytes_per_cell_word" in d and n is not None and mean_words is not None:
        return float(d["dram_bytes_per_cell_word"]) * n * mean_words, (
            d.get("capture", "") + f" (captured on {d['cells']} cells at rank {d['rank']}; scaled to {n} cells and "
            f"{mean_words:.1f} words per cell)")
    return float(d["dram_bytes_per_launch"]), d.get("capture", "")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region (samples go
    to a temporary file that is removed afterwards)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="bench_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _start_ranks(log):
    """Rank at the start of every energy step of one solve from its rank log."""
    K = len(log)
    r_start = np.zeros(K, dtype=np.int64)
    for k in range(1, K):
        a, b = log[k - 1]
        r_start[k] = b if b >= 0 else max(a, 0)
    return r_start


def stage_work(cfg, r_start, nsub):
    """Algorithmic bytes and flops of the streaming-stage launches of one solve: per cell and
    launch (5r + 1) words (stage input, state and output columns of K, the next stage's scaled
    input, rho^-1) and 2 nk r^2 + 6 nk r flops (the r x r mix of nk stencils and the stencils)."""
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    nk = 4 if cfg["ny"] == 1 and cfg["dy"] == 0 else 6
    esize = 8 if cfg["precision"] == 0 else 4
    act = r_start > 0
    launches = 4 * np.asarray(nsub)[act]
    r = r_start[act].astype(np.float64)
    byts = float(np.sum(launches * n * (5 * r + 1) * esize))
    flops = float(np.sum(launches * n * (2 * nk * r * r + 6 * nk * r)))
    return int(np.sum(launches)), byts, flops


def _oracle_block(cfg, mats, w, edge):
    """The central edge^3 block of a 3-D workload's grid (same voxels and mixture weights)."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    i0, j0, k0 = (nx - edge) // 2, (ny - edge) // 2, 0
    W = np.asarray(w).reshape(len(mats), nz, ny, nx)[:, k0:k0 + edge, j0:j0 + edge, i0:i0 + edge]
    c = dict(cfg, nx=edge, ny=edge, nz=edge)
    return c, W.reshape(len(mats), -1), (i0 * cfg["dx"], j0 * cfg["dy"], k0 * cfg["dz"])


def _oracle_step_seconds(cfg, mats, w, beams, edge, k0, reps):
    """Seconds of one FP64 oracle energy step k0 on the central edge^3 block of the workload, from a
    state at the workload's rank (random orthonormal factors, decaying singular values), the source
    of the workload's beam traced through the block; returns (times, the block's n_sub at k0)."""
    from oracle import dlra as ODL
    from oracle import problem as OP
    from oracle import raytrace as ORT
    c, wb, off = _oracle_block(cfg, mats, w, edge)
    prob = OP.Problem(c, mats, wb)
    b = dict(beams[0])
    b["pos"] = [b["pos"][0] - off[0], b["pos"][1] - off[1], b["pos"][2] - off[2]]
    b["spot_sigma"] = min(float(b.get("spot_sigma", 0.0)), 0.1)
    r = ORT.trace(prob, b)
    src = [(r.psi, r.e_u, np.asarray(b["dir"]))]
    rank = int(cfg["rank_max"])
    times = []
    for rep in range(reps):
        rng = np.random.default_rng(rep)
        st = ODL.State(prob.n, prob.m)
        st.X = np.linalg.qr(rng.standard_normal((prob.n, rank)))[0]
        st.W = np.linalg.qr(rng.standard_normal((prob.m, rank)))[0]
        st.S = np.diag(1e-3 * 0.9 ** np.arange(rank))
        rc = ODL.RankControl(mode=OP.FIXED, rank=rank, r_max=rank)
        t0 = time.perf_counter()
        ODL.step(prob, st, k0, src, rc)
        times.append(time.perf_counter() - t0)
    return times, prob.n_sub(k0)


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baseline(name, edge=16, k0=60, reps=2, one_core=True):
    """The FP64 oracle as it stands, on the host cores: energy step k0 of the workload on its central
    edge^3 block, scaled to the whole grid by the cell count and the sub-step count of step k0."""
    cfg, mats, w, beams = _workload(name)
    from oracle import problem as OP
    prob_full_nsub = OP.Problem(cfg, mats, w).n_sub(k0)
    times, nsub_b = _oracle_step_seconds(cfg, mats, w, beams, edge, k0, reps)
    n_full = cfg["nx"] * cfg["ny"] * cfg["nz"]
    scale = n_full / edge ** 3 * prob_full_nsub / max(nsub_b, 1)
    out = {"value": 1.0 / (min(times) * scale), "unit": UNIT, "cores": _cores(), "kind": "oracle",
           "min_s": min(times), "median_s": float(np.median(times)), "runs": reps,
           "sample": f"energy step {k0} of {name} on its central {edge}^3 block (FP64 oracle, rank "
                     f"{cfg['rank_max']} state, {nsub_b} RK4 sub-steps), scaled by the cell count "
                     f"({n_full}/{edge ** 3}) and the workload's sub-steps at that step ({prob_full_nsub}); "
                     f"min of {reps} runs, numpy/BLAS threads on {_cores()} cores"}
    if one_core:
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "t, nb = bench._oracle_step_seconds(*bench._workload(%r), %d, %d, 1); print(json.dumps([t, nb]))"
                % (ROOT, name, edge, k0))
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        try:
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
            t1, _ = json.loads(r.stdout.strip().splitlines()[-1])
            out["one_core"] = {"value": 1.0 / (min(t1) * scale), "seconds": min(t1)}
        except Exception as e:  # the 1-core figure is context only
            out["one_core"] = {"error": str(e)[:200]}
    return out


def _solve_dose(cfg, mats, w, beams, K, lanes, graphs):
    """Device time (ms) of one whole solve after a warm-up solve, and its dose."""
    import torch
    from paper_2508_04484_gb300 import dlra as D
    stream = torch.cuda.Stream()
    s = D.Solver(dict(cfg, max_concurrent_beams=lanes), mats, w, beams, stream=stream.cuda_stream)
    s.autotune()
    s.set_graphs(graphs)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    dose = torch.zeros(n, dtype=torch.float64, device="cuda")
    ms = 0.0
    for i in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.reset(retrace=True)
        s.step(K)
        s.dose(out=dose)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    s.close()
    return ms, dose.cpu().numpy()


def _plain_vs_batched(cfg, mats, w, beams, K, args=None, with_direct=False):
    """The same multi-beam solve with one beam after the other (one lane, direct launches) and
    with the beams advanced concurrently (one lane per beam, energy steps replayed from a CUDA
    graph); one warm-up solve each, then one timed solve; the doses must agree."""
    lanes = min(len(beams), 32)
    plain, d_plain = _solve_dose(cfg, mats, w, beams, K, 1, False)
    graph, d_graph = _solve_dose(cfg, mats, w, beams, K, lanes, True)
    out = {"plain_ms_per_solve": plain, "batched_ms_per_solve": graph, "speedup": plain / graph,
           "beams": len(beams), "lanes": lanes, "energy_steps": K,
           "dose_rel_diff": float(np.linalg.norm(d_graph - d_plain) / np.linalg.norm(d_plain)),
           "batched": "one lane (work space + stream pair) per beam, energy steps replayed from a CUDA graph",
           "plain": "one beam after the other, direct launches"}
    if with_direct:
        out["batched_direct_launch_ms_per_solve"], _ = _solve_dose(cfg, mats, w, beams, K, lanes, False)
    return out


def _batched_line(name="phantom_64cube_8beams"):
    """Batched against plain per-beam solves of a multi-beam workload (the 64^3 eight-beam
    phantom with beam weights U(0.5, 1.5)), with the batched solve's energy steps per second."""
    cfg, mats, w, beams = _workload(name)
    K = cfg["n_steps"]
    r = _plain_vs_batched(cfg, mats, w, beams, K)
    r["workload"] = name
    r["config"] = _config_block(name, cfg, beams, K)
    r["value"] = K / (r["batched_ms_per_solve"] / 1000.0)
    r["unit"] = UNIT
    r["beam_energy_steps_per_s"] = r["value"] * len(beams)
    return r


def _config_block(name, cfg, beams, K):
    return {"workload": name, "voxels": f"{cfg['nx']}x{cfg['ny']}x{cfg['nz']}", "voxel_mm": 10.0 * cfg["dx"],
            "beams": len(beams), "beam_MeV": [round(b["energy"], 1) for b in beams][:4],
            "collision": "boltzmann screened-Rutherford + ETC" if cfg["collision"] == 1 else "fokker-planck",
            "sh_degree": cfg["N"], "moments": (cfg["N"] + 1) ** 2,
            "rank": ("adaptive tol %g, max %d" % (cfg["trunc_tol"], cfg["rank_max"])) if cfg["rank_mode"] == 1
            else "fixed %d" % cfg["rank"],
            "energy_steps": K, "precision": PRECISION_NAMES[cfg["precision"]]}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    name = args.workload
    cfg, mats, w, beams = _workload(name)
    from oracle import problem as OP
    edge, k0 = 12, 60
    nsub_full = OP.Problem(cfg, mats, w).n_sub(k0)
    n_full = cfg["nx"] * cfg["ny"] * cfg["nz"]
    samples = []
    nsub_b = 1
    for i in range(args.warmup + args.steps):
        t, nsub_b = _oracle_step_seconds(cfg, mats, w, beams, edge, k0, 1)
        if i >= args.warmup:
            samples.append(t[0])
    scale = n_full / edge ** 3 * nsub_full / max(nsub_b, 1)
    val = float(args.steps / (np.sum(samples) * scale))
    sample = (f"each step: energy step {k0} of {name} on its central {edge}^3 block (FP64 oracle, rank "
              f"{cfg['rank_max']} state, {nsub_b} RK4 sub-steps), scaled by the cell count ({n_full}/{edge ** 3}) "
              f"and the workload's sub-steps at that step ({nsub_full}); numpy/BLAS threads on {_cores()} cores")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / val, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(_config_block(name, cfg, beams, cfg["n_steps"]), precision="FP64 (oracle)",
                           reference_sample=sample),
            "cpu_baseline": {"value": val, "unit": UNIT, "kind": "oracle", "cores": _cores(), "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _second_line(args, stream):
    """Whole solves of the 64^3 water workload (P_15, rank 20) at the FP32-split precision."""
    import torch
    from paper_2508_04484_gb300 import dlra as D
    cfg, mats, w, beams = _workload(SECOND)
    cfg = dict(cfg, precision=2)
    s = D.Solver(cfg, mats, w, beams, stream=stream.cuda_stream)
    tuned = s.autotune() if not args.no_autotune else None
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    dose = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    K = cfg["n_steps"]
    times = []
    with torch.cuda.stream(stream):
        for i in range(5):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.reset(retrace=True)
            s.step(K)
            s.dose(out=dose)
            e1.record(stream)
            e1.synchronize()
            if i >= 2:
                times.append(e0.elapsed_time(e1))
    s.close()
    ms = float(np.mean(times))
    return {"workload": SECOND, "value": K / (ms / 1000.0), "unit": UNIT, "ms_per_solve": ms,
            "config": _config_block(SECOND, cfg, beams, K), "steps": "3 whole solves after 2 warm-up solves",
            "stage_variant": tuned["stage_variant"] if tuned else None}


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2508_04484_gb300 import build as B
    from paper_2508_04484_gb300 import dlra as D
    B.build()
    name = args.workload
    cfg, mats, w, beams = _workload(name)
    if args.precision is not None:
        cfg = dict(cfg, precision=args.precision)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    K = cfg["n_steps"] if args.energy_steps <= 0 else min(args.energy_steps, cfg["n_steps"])
    steps = max(1, args.steps)
    chunk = max(1, math.ceil(K / steps))
    vs_plain = None
    if len(beams) > 1 and ws == 1:
        vs_plain = _plain_vs_batched(cfg, mats, w, beams, K, args)
    elif ws == 1 and not args.no_batched and name == WORKLOAD:
        vs_plain = _batched_line()
    stream = torch.cuda.Stream(device=dev)
    # several ranks and several beams: each rank solves its share of the plan (beams are
    # independent) and the deposits are summed at the end of every solve; otherwise every rank
    # solves the whole workload (replicas, weak scaling)
    from paper_2508_04484_gb300 import multigpu as MG
    shard = ws > 1 and len(beams) > 1 and not args.replicas
    my_beams = MG.shard_beams(beams, rank, ws) if shard else beams
    solver = D.Solver(dict(cfg, max_concurrent_beams=min(len(my_beams), 32)), mats, w, my_beams,
                      stream=stream.cuda_stream)
    nsub = solver.substeps()[:K]
    dose = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    cursor = [0]

    def bench_step():
        """The next chunk of energy steps of the current solve (a new solve starts with a reset and
        ray trace, the last chunk of a solve ends with the dose read)."""
        if cursor[0] == 0:
            solver.reset(retrace=True)
        ne = min(chunk, K - cursor[0])
        solver.step(ne)
        cursor[0] += ne
        if cursor[0] >= K:
            solver.dose(out=dose)
            if shard:
                MG.reduce_dose(dose)
            cursor[0] = 0
        return ne

    tuned = solver.autotune() if not args.no_autotune else None
    if args.stage_kernel is not None:
        solver.set_stage_kernel(args.stage_kernel)
    if args.stencil_gram_kernel is not None:
        solver.set_stencil_gram_kernel(args.stencil_gram_kernel)
    if args.apply_kernel is not None:
        solver.set_apply_kernel(args.apply_kernel)
    if args.gram_kernel is not None:
        solver.set_gram_kernel(args.gram_kernel)
    # the kernels the timed solver runs, applied again to the end-to-end solver (a user tunes once
    # and sets the chosen kernels on later contexts)
    chosen = {
        "stage": args.stage_kernel if args.stage_kernel is not None else (
            STAGE_NAMES.get(tuned["stage_variant"], 0) if tuned else None),
        "stencil_gram": args.stencil_gram_kernel if args.stencil_gram_kernel is not None else (
            GRAM_NAMES.get(tuned["stencil_gram_kernel"], 0) if tuned else None),
        "apply": args.apply_kernel if args.apply_kernel is not None else (
            APPLY_NAMES.get(tuned["apply_kernel"], 0) if tuned else None),
        "gram": args.gram_kernel if args.gram_kernel is not None else (
            APPLY_NAMES.get(tuned["gram_kernel"], 0) if tuned else None),
    }
    use_graphs = args.graphs == "on" or (args.graphs == "auto" and len(beams) > 1)
    solver.set_graphs(use_graphs)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            bench_step()
        while cursor[0] != 0:      # finish the warm-up solve: the timed steps start a new solve
            bench_step()
    torch.cuda.synchronize()
    log = solver.rank_log(0)[:K]
    r_start = _start_ranks(log)
    updates = int(np.sum(r_start) * n)
    # the ray trace alone (part of the first timed step): a reset with a fresh trace, best of three
    rt_ms = []
    for _ in range(3):
        t0 = time.perf_counter()
        solver.reset(retrace=True)
        torch.cuda.synchronize()
        rt_ms.append((time.perf_counter() - t0) * 1000.0)
    raytrace_ms = min(rt_ms)
    cursor[0] = 0
    clocks = Clocks(dev.index)
    # ---- timed region: K bench steps = whole solves, L2 flushed between steps ----
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # per-launch events of the stage kernel inside the timed region; graph replay hides
    # individual kernels, so with graphs they come from one profiled solve afterwards
    solver.set_profiling(not use_graphs)
    launches0 = solver.launch_count()
    times, esteps = [], 0
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            esteps += bench_step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    launches = solver.launch_count() - launches0
    if use_graphs:
        solver.set_profiling(True)
        with torch.cuda.stream(stream):
            solver.reset(retrace=True)
            solver.step(K)
        torch.cuda.synchronize()
    stage_ms, stage_count = solver.kernel_stats()
    solver.set_profiling(False)
    total_ms = float(np.sum(times))
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    solves = esteps / K
    value = (1 if shard else ws) * esteps / (total_ms / 1000.0)
    updates_per_s = (1 if shard else ws) * updates * solves / (total_ms / 1000.0)
    # ---- roofline of the dominant kernel: fused streaming stage (stencil x r-by-r mix) ----
    nl_solve, bytes_solve, flops_solve = stage_work(cfg, r_start, nsub)
    avg_launch_ms = stage_ms / max(stage_count, 1)
    avg_bytes = bytes_solve / max(nl_solve, 1)
    avg_flops = flops_solve / max(nl_solve, 1)
    peaks, src = _peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12  # FFMA, TFLOP/s
    gbs = avg_bytes / (avg_launch_ms / 1000.0) / 1e9
    tfs = avg_flops / (avg_launch_ms / 1000.0) / 1e12
    frac_hbm = gbs / hbm_peak
    frac_alu = tfs / fp32_peak
    variant = args.stage_kernel if args.stage_kernel is not None else (
        STAGE_NAMES.get(tuned["stage_variant"], 0) if tuned else 0)
    if variant == 3 and cfg["nx"] % 2:
        variant = 0
    esize = 8 if cfg["precision"] == 0 else 4
    traffic, traffic_note = _stage_traffic(variant, name, n, avg_bytes / (n * esize))
    traffic_gbs = traffic / (avg_launch_ms / 1000.0) / 1e9 if traffic else None
    kname = f"{STAGE_KERNELS[variant][0]} (fused RK4 streaming stage: stencil + r x r mix)"
    common = {"traffic": traffic, "traffic_note": traffic_note, "algorithmic_bytes_per_launch": avg_bytes,
              "algorithmic_flops_per_launch": avg_flops, "kernel": kname, "launches_per_solve": nl_solve,
              "avg_launch_us": avg_launch_ms * 1000.0,
              "durations": "profiled solve after the timed region (graph replay)" if use_graphs else "timed region",
              "traffic_gbs": traffic_gbs, "traffic_hbm_frac": traffic_gbs / hbm_peak if traffic_gbs else None,
              "counts": "per cell and launch (5r + 1) words and 2 nk r^2 + 6 nk r flops at the step's rank"}
    if variant in (1, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13):
        # the r x r mix on the tensor cores (kind::tf32, three products per FP32-accurate product):
        # the dense TF32 peak from the measured sustained bf16 GEMM rate x the nominal TF32/bf16 ratio
        bf16 = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
        tf32_peak = bf16 * 1.1 / 2.25
        frac_tc = tfs / tf32_peak
        if frac_tc >= frac_hbm:
            roof = dict({"bound": "tensor", "achieved": tfs, "peak": tf32_peak, "unit": "TFLOP/s", "frac": frac_tc,
                         "peak_source": f"{src} sustained bf16 {bf16} TFLOP/s x nominal tf32/bf16 1.1/2.25",
                         "achieved_gbs": gbs, "hbm_frac": frac_hbm, "fp32_fma_frac": frac_alu}, **common)
        else:
            roof = dict({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": frac_hbm,
                         "peak_source": f"{src} hbm_gbs", "achieved_tflops": tfs, "tensor_frac": frac_tc,
                         "tensor_peak_tflops": tf32_peak, "fp32_fma_frac": frac_alu}, **common)
    elif frac_alu >= frac_hbm:
        roof = dict({"bound": "alu", "achieved": tfs, "peak": fp32_peak, "unit": "TFLOP/s", "frac": frac_alu,
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {mhz} MHz ({src} clock)",
                     "achieved_gbs": gbs, "hbm_frac": frac_hbm}, **common)
    else:
        roof = dict({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": frac_hbm,
                     "peak_source": f"{src} hbm_gbs", "achieved_tflops": tfs, "alu_frac": frac_alu}, **common)
    # ---- end to end through the public API with host buffers ----
    e2e = None
    if (rank == 0 or ws > 1) and not args.no_e2e:
        w_host = np.ascontiguousarray(w, dtype=np.float64)
        dose_host = np.zeros(n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = D.Solver(cfg, mats, w_host, my_beams, stream=stream.cuda_stream)
        if chosen["stage"] is not None:
            s2.set_stage_kernel(chosen["stage"])
        if chosen["stencil_gram"] is not None:
            s2.set_stencil_gram_kernel(chosen["stencil_gram"])
        if chosen["apply"] is not None:
            s2.set_apply_kernel(chosen["apply"])
        if chosen["gram"] is not None:
            s2.set_gram_kernel(chosen["gram"])
        s2.set_graphs(use_graphs)
        s2.step(K)
        s2.dose(out=dose_host)
        e2e_s = time.perf_counter() - t0
        s2.close()
        e2e = {"value": (1 if shard else ws) * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(w_host.nbytes),
               "d2h_bytes_per_step": int(dose_host.nbytes),
               "includes": "context creation with angular tables, host->device mixture weights, ray trace, "
                           "all energy steps, dose read back to host (one whole solve) with the kernels the "
                           "timed solver runs"}
    second = None
    if rank == 0 and ws == 1 and not args.no_second and name == WORKLOAD:
        second = _second_line(args, stream)
    # ---- reverse sweep of the 64^3 water workload (gradients of L = |e|^2 / 2), outside the timed region ----
    adj = None
    if rank == 0 and ws == 1 and not args.no_adjoint:
        cfg3, mats3, w3, beams3 = _workload(SECOND)
        K3 = cfg3["n_steps"]
        interval = 16
        s3 = D.Solver(cfg3, mats3, w3, beams3, stream=stream.cuda_stream)
        s3.enable_adjoint(interval)
        n3 = cfg3["nx"] * cfg3["ny"] * cfg3["nz"]
        g_dev = torch.zeros(n3, dtype=torch.float64, device=dev)
        dw_dev = torch.empty((len(mats3), n3), dtype=torch.float64, device=dev)
        fwd, bwd = [], []
        for _ in range(2):
            s3.reset(retrace=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s3.step(K3)
            s3.dose(out=g_dev)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s3.backward(g_dev, dw_out=dw_dev)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            fwd.append(t1 - t0)
            bwd.append(t2 - t1)
        s3.close()
        adj = {"workload": SECOND, "ms_per_backward": 1000.0 * min(bwd),
               "ms_forward_with_checkpoints": 1000.0 * min(fwd), "backward_over_forward": min(bwd) / min(fwd),
               "checkpoint_interval": interval, "loss": "|e|^2/2 (dL/de = e)",
               "outputs": "dL/dweight per beam, dL/dw per material and cell",
               "timing": "host wall clock around synchronising calls, best of two passes"}
    cb = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and len(beams) == 1 and cfg["ny"] > 1:
        cb = cpu_baseline(name)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
                "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
                "scaling": "strong" if shard else "weak",
                "vs_baseline": None, "dtype": "f64" if cfg["precision"] == 0 else "f32+f64", "data": "synthetic",
                "config": dict(_config_block(name, cfg, beams, K),
                               step=f"{chunk} consecutive energy steps of the solve; {steps} steps = "
                                    f"{solves:g} whole solve(s) (ray trace, {K} energy steps, dose read)",
                               l2="flushed (256 MB write) between timed steps; the factors exceed L2"),
                "cell_rank_updates_per_s": updates_per_s,
                "energy_steps_per_s": value,
                "ms_per_solve": total_ms / solves,
                "gpu_launches": int(launches),
                "roofline": roof, "clocks": ck, "e2e": e2e, "cpu_baseline": cb,
                "vs_plain": vs_plain, "second": second, "adjoint": adj, "cuda_graphs": use_graphs,
                "autotune": tuned,
                "ranks": {"mean": float(np.mean(r_start)), "max": int(np.max(r_start))},
                "raytrace_ms": {"value": raytrace_ms, "timing": "host wall clock around a reset with a fresh "
                                "ray trace of every beam and a synchronise, best of three; inside the first step"}}
        if len(beams) > 1:
            line["beam_energy_steps_per_s"] = value * len(beams)
        print(json.dumps(line))
    solver.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
