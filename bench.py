"""Throughput of the low-rank collided-proton transport solve on GB300.

One bench step is one whole transport solve of the workload: the CSDA ray trace
of the beam, every energy step of the low-rank integrator (streaming BUG with RK4,
implicit collided scattering, first-collision source, truncations) and the dose.
Default workload: 64^3 voxels of 2 mm water, one 150 MeV pencil beam, Boltzmann
screened-Rutherford scattering (eta = 1e-3, extended transport correction),
P_15 (256 moments), fixed rank 20, 200 energy steps 150 -> 1 MeV, FP32 n-side
arithmetic with FP64 reductions/factorisations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores, each step a bounded
sample (a few energy steps) of the same workload. Under torchrun each rank runs
its own copy of the workload (beams are independent: weak scaling); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "energy steps/s and cell·rank updates/s per GB300, % HBM roofline, vs plain"
UNIT = "energy steps/s"
WORKLOAD = "water_64cube_boltzmann"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-adjoint", action="store_true", help="skip timing the reverse sweep (dlra_backward)")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch variants")
    p.add_argument("--stage-kernel", type=int, choices=[0, 1, 2, 3], default=None,
                   help="profiling: streaming-stage kernel (0 per-cell FMA, 1 tensor cores, 2 brick, 3 cell pairs), "
                        "set after the autotuner")
    p.add_argument("--stencil-gram-kernel", type=int, choices=[0, 1], default=None,
                   help="profiling: stencil-Gram kernel (0 FMA, 1 tensor cores), set after the autotuner")
    p.add_argument("--replicas", action="store_true",
                   help="with several ranks, solve the whole multi-beam workload on every rank")
    p.add_argument("--graphs", default="auto", choices=["auto", "on", "off"],
                   help="replay the energy steps from CUDA graphs (auto: on for multi-beam workloads)")
    p.add_argument("--energy-steps", type=int, default=0,
                   help="profiling only: stop each solve after this many energy steps")
    p.add_argument("--workload", default=WORKLOAD,
                   choices=[WORKLOAD, "phantom_48cube_8beams", "phantom_96cube_32beams", "phantom_128cube_adaptive"])
    return p.parse_args()


def _workload(name=WORKLOAD):
    from paper_2508_04484_gb300 import workloads as WL
    return getattr(WL, name)()


# streaming-stage kernels by variant: name and the markers of their source text in device.cuh
# (the DRAM traffic of a capture is reported only while that text is unchanged)
STAGE_KERNELS = {
    0: ("kstage_kernel", "template <typename T, int RM, int NACT>\n__global__ void __launch_bounds__(128) kstage_kernel(",
        "// The streaming stage of kstage_kernel on the FP32 path with two"),
    1: ("kstage_tc_kernel", None, None),
    2: ("kstage_brick_kernel", "// Cell bricks of the staged streaming stage", None),
    3: ("kstage_pair_kernel", "// The streaming stage of kstage_kernel on the FP32 path with two",
        "// Cell bricks of the staged streaming stage"),
}
STAGE_NAMES = {"per-cell FMA": 0, "tensor cores": 1, "brick FMA": 2, "cell pairs": 3}


def stage_source_sha256(variant):
    """sha256 of the source text of a streaming-stage kernel, or None without markers."""
    import hashlib
    _, begin, end = STAGE_KERNELS[variant]
    if begin is None or end is None:
        return None
    src = open(os.path.join(ROOT, "paper_2508_04484_gb300", "csrc", "device.cuh")).read()
    i = src.find(begin)
    j = src.find(end, i + 1) if i >= 0 else -1
    if i < 0 or j < i:
        return None
    return hashlib.sha256(src[i:j].encode()).hexdigest()


def _stage_traffic(variant):
    """DRAM bytes per launch of the streaming-stage kernel in use from the committed ncu summary,
    or None when there is none or the kernel's source changed since that capture."""
    name = STAGE_KERNELS[variant][0]
    path = os.path.join(ROOT, "profiles", "kstage_traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f).get("kernels", {}).get(name)
    if d is None:
        return None, f"no capture of {name}"
    h = stage_source_sha256(variant)
    if h is None or d.get("source_sha256") != h:
        return None, "kernel changed since the capture"
    return float(d["dram_bytes_per_launch"]), d.get("capture", "")


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
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
        for line in open(self.path):
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


def _rank_stats(log, nsub, n):
    """Cell-rank updates and streaming-stage work of one solve from its rank log."""
    K = len(nsub)
    r_start = np.zeros(K, dtype=np.int64)
    for k in range(1, K):
        a, b = log[k - 1]
        r_start[k] = b if b >= 0 else max(a, 0)
    updates = int(np.sum(r_start) * n)
    active = r_start > 0
    stage_launches = int(np.sum(4 * np.asarray(nsub)[active]))
    return r_start, updates, stage_launches


def cpu_baseline(cfg, mats, w, beams, budget_steps=1, k0=40):
    """The FP64 oracle as it stands, on the host cores, for energy steps k0, k0 + 1, ... of the
    workload started from a state at the workload's full rank (random orthonormal factors,
    decaying singular values): the steady-state cost of a step, which most of the 200 steps pay
    (the first steps, at rank 1-10, are far cheaper). Source from a single central ray."""
    from oracle import dlra as ODL
    from oracle import problem as OP
    from oracle import raytrace as ORT
    prob = OP.Problem(cfg, mats, w)
    b = dict(beams[0], spot_sigma=0.0)
    r = ORT.trace(prob, b)
    src = [(r.psi, r.e_u, np.asarray(b["dir"]))]
    rank = int(cfg["rank"])
    rng = np.random.default_rng(0)
    st = ODL.State(prob.n, prob.m)
    st.X = np.linalg.qr(rng.standard_normal((prob.n, rank)))[0]
    st.W = np.linalg.qr(rng.standard_normal((prob.m, rank)))[0]
    st.S = np.diag(1e-3 * 0.8 ** np.arange(rank))
    rc = ODL.RankControl(mode=cfg["rank_mode"], rank=cfg["rank"], tol=cfg["trunc_tol"], r_max=cfg["rank_max"])
    t0 = time.perf_counter()
    upd = 0
    for k in range(k0, k0 + budget_steps):
        upd += prob.n * st.r
        ODL.step(prob, st, k, src, rc)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": budget_steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cell_rank_updates_per_s": upd / dt,
            "sample": f"energy steps {k0}..{k0 + budget_steps - 1} of {WORKLOAD} from a rank-{rank} state "
                      f"(source of one central ray), {dt:.1f} s, numpy/BLAS threads on {cores} cores"}


def _solve_ms(cfg, mats, w, beams, K, lanes, reps, graphs=False):
    """Mean device time (ms) of one whole solve with the given number of lanes (graphs: the
    energy steps replayed from a CUDA graph captured on the first, untimed solve)."""
    import torch
    from paper_2508_04484_gb300 import dlra as D
    stream = torch.cuda.Stream()
    s = D.Solver(dict(cfg, max_concurrent_beams=lanes), mats, w, beams, stream=stream.cuda_stream)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    dose = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.set_graphs(graphs)
    times = []
    for i in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.reset(retrace=True)
        s.step(K)
        s.dose(out=dose)
        e1.record(stream)
        e1.synchronize()
        if i > 0:
            times.append(e0.elapsed_time(e1))
    s.close()
    return float(np.mean(times))


def _plain_vs_batched(cfg, mats, w, beams, K, args):
    """The same multi-beam solve with one beam after the other (one lane) and with the
    beams advanced concurrently (one lane per beam)."""
    reps = max(1, min(args.steps, 3))
    lanes = min(len(beams), 32)
    plain = _solve_ms(cfg, mats, w, beams, K, 1, reps)
    direct = _solve_ms(cfg, mats, w, beams, K, lanes, reps)
    graph = _solve_ms(cfg, mats, w, beams, K, lanes, reps, graphs=True)
    return {"plain_ms_per_solve": plain, "batched_ms_per_solve": graph, "speedup": plain / graph,
            "batched_direct_launch_ms_per_solve": direct, "beams": len(beams), "lanes": lanes,
            "batched": "one lane (work space + stream pair) per beam, energy steps replayed from a CUDA graph"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    cfg, mats, w, beams = _workload()
    samples = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(cfg, mats, w, beams, budget_steps=1)
        if i >= args.warmup:
            samples.append(cb)
    val = float(np.mean([s["value"] for s in samples]))
    ms = 1000.0 / val * cfg["n_steps"]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "voxels": "64x64x64", "voxel_mm": 2.0, "sh_degree": 15,
                       "rank": 20, "energy_steps": 200, "beams": 1,
                       "reference_sample": "each step: one energy step of the FP64 oracle at full rank"},
            "cpu_baseline": {"value": val, "unit": UNIT, "kind": "oracle", "cores": samples[0]["cores"],
                             "sample": samples[0]["sample"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


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
    cfg, mats, w, beams = _workload(args.workload)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    K = cfg["n_steps"] if args.energy_steps <= 0 else min(args.energy_steps, cfg["n_steps"])
    vs_plain = None
    if len(beams) > 1 and ws == 1:
        vs_plain = _plain_vs_batched(cfg, mats, w, beams, K, args)
    stream = torch.cuda.Stream(device=dev)
    # several ranks and several beams: each rank solves its share of the plan (beams are
    # independent) and the deposits are summed at the end of every solve; otherwise every rank
    # solves the whole workload (replicas, weak scaling)
    from paper_2508_04484_gb300 import multigpu as MG
    shard = ws > 1 and len(beams) > 1 and not args.replicas
    my_beams = MG.shard_beams(beams, rank, ws) if shard else beams
    solver = D.Solver(dict(cfg, max_concurrent_beams=min(len(my_beams), 32)), mats, w, my_beams,
                      stream=stream.cuda_stream)
    nsub = solver.substeps()
    dose = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def one_solve():
        solver.reset(retrace=True)
        solver.step(K)
        solver.dose(out=dose)
        if shard:
            MG.reduce_dose(dose)

    tuned = solver.autotune() if not args.no_autotune else None
    if args.stage_kernel is not None:
        solver.set_stage_kernel(args.stage_kernel)
    if args.stencil_gram_kernel is not None:
        solver.set_stencil_gram_kernel(args.stencil_gram_kernel)
    use_graphs = args.graphs == "on" or (args.graphs == "auto" and len(beams) > 1)
    solver.set_graphs(use_graphs)
    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    log = solver.rank_log(0)[:K]
    nsub = nsub[:K]
    r_start, updates, stage_launches = _rank_stats(log, nsub, n)
    # the ray trace alone (part of every timed solve): reset with a fresh trace, best of three
    # (after the rank log of the warm-up solve is read: a reset clears it; every timed solve
    # starts with the same reset)
    rt_ms = []
    for _ in range(3):
        t0 = time.perf_counter()
        solver.reset(retrace=True)
        torch.cuda.synchronize()
        rt_ms.append((time.perf_counter() - t0) * 1000.0)
    raytrace_ms = min(rt_ms)
    clocks = Clocks(dev.index)
    # ---- timed region: K whole solves, L2 flushed between them ----
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # per-launch events of the stage kernel inside the timed region; graph replay hides
    # individual kernels, so with graphs they come from one profiled solve afterwards
    solver.set_profiling(not use_graphs)
    launches0 = solver.launch_count()
    times = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_solve()
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
            one_solve()
        torch.cuda.synchronize()
    stage_ms, stage_count = solver.kernel_stats()
    solver.set_profiling(False)
    ms_per_solve = float(np.sum(times) / args.steps)
    if ws > 1:
        t = torch.tensor([ms_per_solve], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_per_solve = float(t.item())
    value = (1 if shard else ws) * K / (ms_per_solve / 1000.0)
    updates_per_s = (1 if shard else ws) * updates / (ms_per_solve / 1000.0)
    # ---- roofline of the dominant kernel: fused streaming stage (stencil x r-by-r mix) ----
    nk = 4 if cfg["ny"] == 1 and cfg["dy"] == 0 else 6
    esize = 4 if cfg["precision"] == 1 else 8
    act = r_start > 0
    per_solve_launches = int(np.sum(4 * np.asarray(nsub)[act]))
    bytes_solve = float(np.sum((4 * np.asarray(nsub) * n * (3 * r_start + 1) * esize)[act]))
    flops_solve = float(np.sum((4 * np.asarray(nsub) * n * 2 * nk * r_start.astype(np.float64) ** 2)[act]))
    avg_launch_ms = stage_ms / max(stage_count, 1)
    avg_bytes = bytes_solve / max(per_solve_launches, 1)
    avg_flops = flops_solve / max(per_solve_launches, 1)
    peaks, src = _peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    fp32_peak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12  # FFMA, TFLOP/s
    gbs = avg_bytes / (avg_launch_ms / 1000.0) / 1e9
    tfs = avg_flops / (avg_launch_ms / 1000.0) / 1e12
    frac_hbm = gbs / hbm_peak
    frac_alu = tfs / fp32_peak
    variant = args.stage_kernel if args.stage_kernel is not None else (
        STAGE_NAMES.get(tuned["stage_variant"], 0) if tuned else 0)
    if variant == 3 and cfg["nx"] % 2:
        variant = 0
    traffic, traffic_note = _stage_traffic(variant)
    # the same launch measured by its DRAM bytes (ncu capture) over its CUDA-event time
    traffic_gbs = traffic / (avg_launch_ms / 1000.0) / 1e9 if traffic else None
    kname = f"{STAGE_KERNELS[variant][0]} (fused RK4 streaming stage: stencil + r x r mix)"
    if frac_alu >= frac_hbm:
        roof = {"bound": "alu", "achieved": tfs, "peak": fp32_peak, "unit": "TFLOP/s", "frac": frac_alu,
                "traffic": traffic, "traffic_note": traffic_note, "algorithmic_bytes_per_launch": avg_bytes,
                "algorithmic_flops_per_launch": avg_flops, "kernel": kname,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz ({src} clock)",
                "durations": "profiled solve after the timed region (graph replay)" if use_graphs else "timed region",
                "achieved_gbs": gbs, "hbm_frac": frac_hbm, "avg_launch_us": avg_launch_ms * 1000.0,
                "traffic_gbs": traffic_gbs, "traffic_hbm_frac": traffic_gbs / hbm_peak if traffic_gbs else None}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": frac_hbm,
                "traffic": traffic, "traffic_note": traffic_note, "algorithmic_bytes_per_launch": avg_bytes,
                "algorithmic_flops_per_launch": avg_flops, "kernel": kname,
                "peak_source": f"{src} hbm_gbs", "achieved_tflops": tfs, "alu_frac": frac_alu,
                "traffic_gbs": traffic_gbs, "traffic_hbm_frac": traffic_gbs / hbm_peak if traffic_gbs else None,
                "durations": "profiled solve after the timed region (graph replay)" if use_graphs else "timed region",
                "avg_launch_us": avg_launch_ms * 1000.0}
    # ---- end to end through the public API with host buffers ----
    e2e = None
    if (rank == 0 or ws > 1) and not args.no_e2e:
        w_host = np.ascontiguousarray(w, dtype=np.float64)
        dose_host = np.zeros(n)
        e2e_times = []
        for i in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = D.Solver(cfg, mats, w_host, my_beams, stream=stream.cuda_stream)
            s2.step(K)
            s2.dose(out=dose_host)
            e2e_times.append(time.perf_counter() - t0)
            s2.close()
        e2e_s = min(e2e_times)
        e2e = {"value": (1 if shard else ws) * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(w_host.nbytes),
               "d2h_bytes_per_step": int(dose_host.nbytes),
               "includes": "context creation with angular tables, host->device mixture weights, ray trace, "
                           "all energy steps, dose read back to host"}
    # ---- reverse sweep (gradients of L = |e|^2 / 2 w.r.t. beam and mixture weights), outside the timed region ----
    adj = None
    if rank == 0 and ws == 1 and not args.no_adjoint:
        interval = 16
        s3 = D.Solver(cfg, mats, w, beams, stream=stream.cuda_stream)
        s3.enable_adjoint(interval)
        g_dev = torch.zeros(n, dtype=torch.float64, device=dev)
        dw_dev = torch.empty((len(mats), n), dtype=torch.float64, device=dev)
        fwd, bwd = [], []
        for _ in range(2):
            s3.reset(retrace=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s3.step(K)
            s3.dose(out=g_dev)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s3.backward(g_dev, dw_out=dw_dev)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            fwd.append(t1 - t0)
            bwd.append(t2 - t1)
        s3.close()
        adj = {"ms_per_backward": 1000.0 * min(bwd), "ms_forward_with_checkpoints": 1000.0 * min(fwd),
               "backward_over_forward": min(bwd) / (ms_per_solve / 1000.0), "checkpoint_interval": interval,
               "loss": "|e|^2/2 (dL/de = e)", "outputs": "dL/dweight per beam, dL/dw per material and cell",
               "timing": "host wall clock around synchronising calls, best of two passes"}
    cb = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cfg_c, mats_c, w_c, beams_c = _workload()
        cb = cpu_baseline(cfg_c, mats_c, w_c, beams_c)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_solve, "higher_is_better": True,
                "scaling": "strong" if shard else "weak",
                "vs_baseline": None, "dtype": "f32+f64" if cfg["precision"] == 1 else "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "voxels": "64x64x64", "voxel_mm": 2.0, "material": "water",
                           "beam_MeV": 150, "collision": "boltzmann screened-Rutherford eta=1e-3 + ETC",
                           "sh_degree": 15, "moments": 256, "rank": 20, "energy_steps": K,
                           "step": "one whole solve (ray trace + all energy steps + dose)",
                           "l2": "flushed (256 MB write) between timed solves"},
                "cell_rank_updates_per_s": updates_per_s,
                "energy_steps_per_s": value,
                "gpu_launches": int(launches),
                "roofline": roof, "clocks": ck, "e2e": e2e, "cpu_baseline": cb,
                "vs_plain": vs_plain, "adjoint": adj, "cuda_graphs": use_graphs, "autotune": tuned,
                "raytrace_ms": {"value": raytrace_ms, "timing": "host wall clock around a reset with a fresh "
                                "ray trace of every beam and a synchronise, best of three; included in each step"}}
        if args.workload != WORKLOAD:
            line["config"] = {"workload": args.workload, "beams": len(beams), "voxels": f"{cfg['nx']}x{cfg['ny']}x{cfg['nz']}",
                              "sh_degree": cfg["N"], "rank_max": cfg["rank_max"], "energy_steps": K,
                              "step": "one whole solve of all beams"}
            line["beam_energy_steps_per_s"] = value * len(beams)
        print(json.dumps(line))
    solver.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
