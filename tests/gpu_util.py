"""Helpers that run the same seeded workload through the oracle and through the C ABI."""
import numpy as np

from oracle import dlra as ODL
from oracle import fullrank as OFR
from oracle import problem as OP
from oracle import raytrace as ORT


def oracle_problem(cfg, mats, w):
    return OP.Problem(cfg, mats, w)


def oracle_sources(prob, beams):
    out = []
    for b in beams:
        r = ORT.trace(prob, b)
        d = np.asarray(b["dir"], float)
        out.append((r.psi, r.e_u, d / np.linalg.norm(d)))
    return out


def oracle_dlra(prob, sources, mode, n_steps=None, **kw):
    """Independent low-rank state per beam (as the library runs them); returns
    (total dose, list of per-beam results)."""
    res = []
    for s in sources:
        rc = ODL.RankControl(mode=mode, **kw)
        res.append(ODL.solve(prob, [s], rc, n_steps=n_steps))
    dose = sum(r["dose"] for r in res)
    return dose, res


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def gpu_solver(cfg, mats, w, beams, schedule=None, precision=None):
    from paper_2508_04484_gb300 import dlra as D
    c = dict(cfg)
    if schedule is not None:
        c["rank_mode"] = OP.SCHEDULE
        c["rank_schedule"] = np.asarray(schedule, dtype=np.int32)
    if precision is not None:
        c["precision"] = precision
    return D.Solver(c, mats, w, beams)
