"""Thin Python binding of the C ABI in ``include/dlra.h``.

Argument marshalling only: every computation runs in the CUDA library
``libdlra.so``. The functions carry the C names; ``Solver`` bundles them for one
context. Device buffers may be given as PyTorch CUDA tensors (their data pointer
is passed with the matching ``*_on_device`` flag); the CUDA stream of a context
is a borrowed ``cudaStream_t`` (e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdlra.so")

DLRA_OK = 0
(DLRA_ERR_ARG, DLRA_ERR_STATE, DLRA_ERR_CUDA, DLRA_ERR_OOM, DLRA_ERR_NONFINITE, DLRA_ERR_RANK,
 DLRA_ERR_TIMEOUT) = range(1, 8)
STATUS = {0: "DLRA_OK", 1: "DLRA_ERR_ARG", 2: "DLRA_ERR_STATE", 3: "DLRA_ERR_CUDA", 4: "DLRA_ERR_OOM",
          5: "DLRA_ERR_NONFINITE", 6: "DLRA_ERR_RANK", 7: "DLRA_ERR_TIMEOUT"}
FOKKER_PLANCK, BOLTZMANN = 0, 1
RANK_FIXED, RANK_ADAPTIVE, RANK_SCHEDULE = 0, 1, 2
FP64, FP32_MIXED, FP32_SPLIT = 0, 1, 2


class DlraError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class dlra_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("sh_degree", C.c_int32), ("collision", C.c_int32), ("transport_correction", C.c_int32),
                ("rank_mode", C.c_int32), ("rank", C.c_int32), ("rank_max", C.c_int32),
                ("trunc_tol", C.c_double), ("rank_schedule", C.POINTER(C.c_int32)),
                ("e_max", C.c_double), ("e_min", C.c_double), ("n_energy_steps", C.c_int32),
                ("cfl_max", C.c_double), ("precision", C.c_int32),
                ("bk_p", C.c_double), ("bk_alpha", C.c_double), ("t100", C.c_double),
                ("max_concurrent_beams", C.c_int32), ("cuda_stream", C.c_void_p)]


class dlra_material(C.Structure):
    _fields_ = [("density", C.c_double), ("sp_ratio", C.c_double), ("scatter_ratio", C.c_double),
                ("screening", C.c_double)]


class dlra_beam(C.Structure):
    _fields_ = [("energy", C.c_double), ("energy_sigma", C.c_double), ("pos", C.c_double * 3),
                ("dir", C.c_double * 3), ("spot_sigma", C.c_double), ("weight", C.c_double)]


class dlra_kstep_args(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("r", C.c_int32), ("e0", C.c_double), ("de", C.c_double), ("n_sub", C.c_int32),
                ("bk_p", C.c_double), ("bk_alpha", C.c_double),
                ("K0", C.c_void_p), ("K1", C.c_void_p), ("inv_rho", C.c_void_p), ("P", C.c_void_p),
                ("cuda_stream", C.c_void_p), ("stage_kernel", C.c_int32)]


class dlra_stencil_gram_args(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("na", C.c_int32), ("nb", C.c_int32),
                ("A", C.c_void_p), ("lda", C.c_int64), ("B", C.c_void_p), ("ldb", C.c_int64),
                ("inv_rho", C.c_void_p), ("out", C.c_void_p), ("variant", C.c_int32),
                ("cuda_stream", C.c_void_p)]


class dlra_straggling_args(C.Structure):
    _fields_ = [("e_min", C.c_double), ("e_max", C.c_double), ("n_elem", C.c_int32),
                ("bk_p", C.c_double), ("bk_alpha", C.c_double), ("t100", C.c_double),
                ("straggling", C.c_int32)]


class dlra_straggling_trace_args(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("e_min", C.c_double), ("e_max", C.c_double), ("n_bins", C.c_int32), ("n_elem", C.c_int32),
                ("h_max", C.c_double), ("bk_p", C.c_double), ("bk_alpha", C.c_double), ("t100", C.c_double),
                ("straggling", C.c_int32), ("energy", C.c_double), ("energy_sigma", C.c_double),
                ("spot_sigma", C.c_double), ("pos", C.c_double * 3), ("dir", C.c_double * 3),
                ("f_cell", C.c_void_p), ("tau_cell", C.c_void_p), ("psi", C.c_void_p), ("e_u", C.c_void_p),
                ("cuda_stream", C.c_void_p)]


# names, argument types and return type of every entry point of include/dlra.h
_P = C.c_void_p
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)
SIGNATURES = {
    "dlra_init": ([C.POINTER(dlra_config), C.POINTER(_P)], C.c_int),
    "dlra_set_materials": ([_P, C.c_int32, C.POINTER(dlra_material), _P, C.c_int32], C.c_int),
    "dlra_add_beam": ([_P, C.POINTER(dlra_beam), _IP], C.c_int),
    "dlra_step": ([_P, C.c_int32], C.c_int),
    "dlra_dose": ([_P, _P, C.c_int32, C.c_int32], C.c_int),
    "dlra_query": ([_P, _IP, _IP], C.c_int),
    "dlra_rank_log": ([_P, C.c_int32, _IP], C.c_int),
    "dlra_get_state": ([_P, C.c_int32, _DP, _DP, _DP, _IP], C.c_int),
    "dlra_set_state": ([_P, C.c_int32, _DP, _DP, _DP, C.c_int32], C.c_int),
    "dlra_get_source": ([_P, C.c_int32, C.c_int32, _DP, _DP], C.c_int),
    "dlra_get_tables": ([_P, _DP, _DP], C.c_int),
    "dlra_get_substeps": ([_P, _IP], C.c_int),
    "dlra_reset": ([_P, C.c_int32], C.c_int),
    "dlra_set_beam_weight": ([_P, C.c_int32, C.c_double], C.c_int),
    "dlra_enable_adjoint": ([_P, C.c_int32], C.c_int),
    "dlra_backward": ([_P, _P, C.c_int32, _DP, _P, C.c_int32], C.c_int),
    "dlra_autotune": ([_P, _DP], C.c_int),
    "dlra_set_stage_kernel": ([_P, C.c_int32], C.c_int),
    "dlra_set_gram_kernel": ([_P, C.c_int32], C.c_int),
    "dlra_set_tensor_cores": ([_P, C.c_int32], C.c_int),
    "dlra_set_graphs": ([_P, C.c_int32], C.c_int),
    "dlra_set_adjoint_store": ([_P, C.c_int32], C.c_int),
    "dlra_set_stencil_gram_kernel": ([_P, C.c_int32], C.c_int),
    "dlra_set_profiling": ([_P, C.c_int32], C.c_int),
    "dlra_kernel_stats": ([_P, _DP, C.POINTER(C.c_int64)], C.c_int),
    "dlra_kstep": ([C.POINTER(dlra_kstep_args)], C.c_int),
    "dlra_kstep_noalloc": ([C.POINTER(dlra_kstep_args)], C.c_int),
    "dlra_set_joint": ([_P, C.c_int32], C.c_int),
    "dlra_set_apply_kernel": ([_P, C.c_int32], C.c_int),
    "dlra_set_straggling": ([_P, C.c_int32, C.c_int32, C.c_double, C.c_int32], C.c_int),
    "dlra_stencil_gram": ([C.POINTER(dlra_stencil_gram_args)], C.c_int),
    "dlra_straggling_tables": ([C.POINTER(dlra_straggling_args), _DP, _DP, _DP, _DP], C.c_int),
    "dlra_straggling_trace": ([C.POINTER(dlra_straggling_trace_args)], C.c_int),
    "dlra_launch_count": ([_P], C.c_int64),
    "dlra_last_error": ([_P], C.c_char_p),
    "dlra_destroy": ([_P], None),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libdlra.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2508_04484_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(ctx, status):
    if status != DLRA_OK:
        msg = load().dlra_last_error(ctx)
        raise DlraError(status, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(_DP)


def _iptr(a):
    return a.ctypes.data_as(_IP)


def make_config(cfg: dict, stream=None):
    c = dlra_config()
    c.nx, c.ny, c.nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"])
    c.dx, c.dy, c.dz = float(cfg["dx"]), float(cfg["dy"]), float(cfg["dz"])
    c.sh_degree = int(cfg["N"])
    coll = cfg["collision"]
    if isinstance(coll, str):
        coll = BOLTZMANN if coll.lower().startswith("b") else FOKKER_PLANCK
    c.collision = int(coll)
    c.transport_correction = int(cfg.get("transport_correction", 1))
    c.rank_mode = int(cfg.get("rank_mode", RANK_FIXED))
    c.rank = int(cfg.get("rank", 5))
    c.rank_max = int(cfg.get("rank_max", max(c.rank, 1)))
    c.trunc_tol = float(cfg.get("trunc_tol", 1e-3))
    c.e_max, c.e_min = float(cfg["e_max"]), float(cfg["e_min"])
    c.n_energy_steps = int(cfg["n_steps"])
    c.cfl_max = float(cfg.get("cfl", 0.6))
    c.precision = int(cfg.get("precision", FP64))
    c.bk_p = float(cfg.get("bk_p", 1.77))
    c.bk_alpha = float(cfg.get("bk_alpha", 0.0022))
    c.t100 = float(cfg.get("t100", 1.72e-4))
    c.max_concurrent_beams = int(cfg.get("max_concurrent_beams", 0))
    c.cuda_stream = stream
    sched = cfg.get("rank_schedule")
    keep = None
    if sched is not None:
        keep = np.ascontiguousarray(np.asarray(sched, dtype=np.int32).reshape(-1))
        c.rank_schedule = _iptr(keep)
    return c, keep


# ---------------------------------------------------------------------------
# functions with the C names
# ---------------------------------------------------------------------------
def dlra_init(cfg: dict, stream=None):
    lib = load()
    c, keep = make_config(cfg, stream)
    h = _P()
    st = lib.dlra_init(C.byref(c), C.byref(h))
    if st != DLRA_OK:
        msg = lib.dlra_last_error(h) if h.value else b"invalid configuration"
        if h.value:
            lib.dlra_destroy(h)
        raise DlraError(st, msg.decode())
    del keep
    return h


def dlra_set_materials(ctx, materials, w):
    mats = (dlra_material * len(materials))()
    for i, m in enumerate(materials):
        mats[i].density = m["density"]
        mats[i].sp_ratio = m.get("sp_ratio", 1.0)
        mats[i].scatter_ratio = m.get("scatter_ratio", 1.0)
        mats[i].screening = m.get("screening", 1e-3)
    if _is_cuda_tensor(w):
        _check(ctx, load().dlra_set_materials(ctx, len(materials), mats, C.c_void_p(w.data_ptr()), 1))
    else:
        wa = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        _check(ctx, load().dlra_set_materials(ctx, len(materials), mats, wa.ctypes.data_as(C.c_void_p), 0))


def dlra_add_beam(ctx, beam: dict) -> int:
    b = dlra_beam()
    b.energy = beam["energy"]
    b.energy_sigma = beam.get("energy_sigma", 0.0)
    for i in range(3):
        b.pos[i] = beam["pos"][i]
        b.dir[i] = beam["dir"][i]
    b.spot_sigma = beam.get("spot_sigma", 0.0)
    b.weight = beam.get("weight", 1.0)
    bid = C.c_int32()
    _check(ctx, load().dlra_add_beam(ctx, C.byref(b), C.byref(bid)))
    return bid.value


def dlra_step(ctx, n_steps: int):
    _check(ctx, load().dlra_step(ctx, int(n_steps)))


def dlra_dose(ctx, n: int = None, out=None, per_mass=False):
    """Dose into ``out`` (torch CUDA tensor or numpy float64) or a new numpy array of length n."""
    if out is not None and _is_cuda_tensor(out):
        _check(ctx, load().dlra_dose(ctx, C.c_void_p(out.data_ptr()), 1, int(per_mass)))
        return out
    if out is None:
        out = np.zeros(n)
    _check(ctx, load().dlra_dose(ctx, out.ctypes.data_as(C.c_void_p), 0, int(per_mass)))
    return out


def dlra_query(ctx, n_beams: int = 0):
    step = C.c_int32()
    ranks = np.zeros(max(n_beams, 1), dtype=np.int32)
    _check(ctx, load().dlra_query(ctx, C.byref(step), _iptr(ranks)))
    return step.value, ranks[:n_beams]


def dlra_rank_log(ctx, beam_id: int, K: int):
    log = np.zeros(2 * K, dtype=np.int32)
    _check(ctx, load().dlra_rank_log(ctx, beam_id, _iptr(log)))
    return log.reshape(K, 2)


RANK_CAPS = (4, 8, 12, 16, 20, 24, 32, 40, 48, 64)


def rank_capacity(rank_max: int) -> int:
    """Column capacity the library allocates for a given rank_max."""
    return next((c for c in RANK_CAPS if c >= rank_max), 64)


def dlra_get_state(ctx, beam_id: int, n: int, m: int, rank_max: int):
    RB = rank_capacity(rank_max)
    X = np.zeros(n * RB)
    S = np.zeros(RB * RB)
    W = np.zeros(m * RB)
    r = C.c_int32()
    _check(ctx, load().dlra_get_state(ctx, beam_id, _dptr(X), _dptr(S), _dptr(W), C.byref(r)))
    r = r.value
    X = X.reshape(RB, n).T[:, :r].copy()
    W = W.reshape(RB, m).T[:, :r].copy()
    S = S.reshape(RB, RB).T[:r, :r].copy()
    return X, S, W


def dlra_set_state(ctx, beam_id: int, X, S, W, rank_max: int):
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    r = X.shape[1]
    RB = rank_capacity(rank_max)
    Xc = np.ascontiguousarray(X.T).reshape(-1)
    Wc = np.ascontiguousarray(W.T).reshape(-1)
    Sc = np.zeros((RB, RB))
    Sc[:r, :r] = S.T
    Sc = np.ascontiguousarray(Sc).reshape(-1)
    _check(ctx, load().dlra_set_state(ctx, beam_id, _dptr(Xc), _dptr(Sc), _dptr(Wc), r))


def dlra_get_source(ctx, beam_id: int, k: int, n: int):
    psi = np.zeros(n)
    e_u = np.zeros(n)
    _check(ctx, load().dlra_get_source(ctx, beam_id, k, _dptr(psi), _dptr(e_u)))
    return psi, e_u


def dlra_get_tables(ctx, m: int):
    A = np.zeros(3 * m * m)
    absA = np.zeros(3 * m * m)
    _check(ctx, load().dlra_get_tables(ctx, _dptr(A), _dptr(absA)))
    return A.reshape(3, m, m), absA.reshape(3, m, m)


def dlra_get_substeps(ctx, K: int):
    out = np.zeros(K, dtype=np.int32)
    _check(ctx, load().dlra_get_substeps(ctx, _iptr(out)))
    return out


def dlra_reset(ctx, retrace=True):
    _check(ctx, load().dlra_reset(ctx, int(bool(retrace))))


def dlra_set_beam_weight(ctx, beam_id: int, weight: float):
    _check(ctx, load().dlra_set_beam_weight(ctx, int(beam_id), float(weight)))


def dlra_enable_adjoint(ctx, checkpoint_interval: int = 16):
    _check(ctx, load().dlra_enable_adjoint(ctx, int(checkpoint_interval)))


def dlra_backward(ctx, dL_de, n_beams: int, n_mat: int, n: int, dw_out=None):
    """Reverse sweep: returns (dL/dweight (n_beams,) numpy, dL/dw (n_mat, n)).

    ``dL_de``: numpy float64 (n,) or a CUDA float64 tensor. dL/dw is written into
    ``dw_out`` (CUDA float64 tensor of n_mat * n) when given, else returned as numpy."""
    dbeta = np.zeros(max(n_beams, 1))
    if _is_cuda_tensor(dL_de):
        gin, gdev = C.c_void_p(dL_de.data_ptr()), 1
    else:
        g = np.ascontiguousarray(np.asarray(dL_de, dtype=np.float64).reshape(-1))
        gin, gdev = g.ctypes.data_as(C.c_void_p), 0
    if dw_out is not None and _is_cuda_tensor(dw_out):
        _check(ctx, load().dlra_backward(ctx, gin, gdev, _dptr(dbeta), C.c_void_p(dw_out.data_ptr()), 1))
        return dbeta[:n_beams], dw_out
    dw = np.zeros((n_mat, n))
    _check(ctx, load().dlra_backward(ctx, gin, gdev, _dptr(dbeta), dw.ctypes.data_as(C.c_void_p), 0))
    return dbeta[:n_beams], dw


def dlra_autotune(ctx):
    """Pick the fastest launch variants on this context; returns the timing report as a dict."""
    rep = np.zeros(31)
    _check(ctx, load().dlra_autotune(ctx, _dptr(rep)))
    return dict(stage_fma_ms=rep[0], stage_tensor_core_ms=rep[1], stage_brick_ms=rep[12],
                gram_ms=dict(zip((608, 1216, 2432, 4864), rep[2:6])),
                stencil_gram_ms=dict(zip((0.5, 1.0, 2.0), rep[6:9])), stencil_gram_tc_ms=rep[13],
                stage_pair_ms=rep[15], stage_tma128_ms=rep[16], stage_tma256_ms=rep[17],
                stage_tma_persistent_ms=rep[18], stage_tma_tmem_a_ms=rep[19], stage_tma_cluster_ms=rep[23], stage_tma_tiles3_ms=rep[25], stage_tma_chunk8_ms=rep[27],
                stage_tma_form8_ms=rep[28], stage_tma_faces_ms=rep[29],
                stage_tma_faces_split_b_ms=rep[30],
                apply_fma_ms=rep[20], apply_tensor_core_ms=rep[21],
                apply_kernel=("FMA", "tensor cores")[int(rep[22])],
                stage_variant=("per-cell FMA", "tensor cores", "brick FMA", "cell pairs", "TMA tensor cores 128",
                               "TMA tensor cores 256", "TMA tensor cores persistent",
                               "TMA tensor cores A in TMEM", "TMA tensor cores cluster",
                               "TMA tensor cores 3 tiles", "TMA tensor cores 8 columns",
                               "TMA tensor cores 8 formation warps", "TMA tensor cores faces",
                               "TMA tensor cores faces split B")[int(rep[9])],
                gram_blocks=int(rep[10]), stencil_gram_waves=rep[11] / 2.0,
                stencil_gram_window_ms=rep[24], gram_tensor_core_ms=rep[26],
                gram_kernel="tensor cores" if 0.0 < rep[26] < min(rep[2:6]) else "FMA",
                stencil_gram_kernel=("FMA", "tensor cores", "tensor cores TMA window")[int(rep[14])])


def dlra_set_stage_kernel(ctx, variant: int):
    _check(ctx, load().dlra_set_stage_kernel(ctx, int(variant)))


def dlra_set_stencil_gram_kernel(ctx, variant: int):
    _check(ctx, load().dlra_set_stencil_gram_kernel(ctx, int(variant)))


def dlra_set_tensor_cores(ctx, enable=True):
    _check(ctx, load().dlra_set_tensor_cores(ctx, int(bool(enable))))


def dlra_set_graphs(ctx, enable=True):
    _check(ctx, load().dlra_set_graphs(ctx, int(bool(enable))))


def dlra_set_straggling(ctx, enable=True, n_elem=128, h_max=0.01, straggling=True):
    _check(ctx, load().dlra_set_straggling(ctx, 1 if enable else 0, int(n_elem), float(h_max), 1 if straggling else 0))


def dlra_set_gram_kernel(ctx, variant: int):
    _check(ctx, load().dlra_set_gram_kernel(ctx, int(variant)))


def dlra_set_apply_kernel(ctx, variant: int):
    _check(ctx, load().dlra_set_apply_kernel(ctx, int(variant)))


def dlra_set_joint(ctx, enable=True):
    _check(ctx, load().dlra_set_joint(ctx, 1 if enable else 0))


def dlra_set_adjoint_store(ctx, keep=True):
    _check(ctx, load().dlra_set_adjoint_store(ctx, int(bool(keep))))


def dlra_set_profiling(ctx, enable=True):
    _check(ctx, load().dlra_set_profiling(ctx, int(bool(enable))))


def dlra_kernel_stats(ctx):
    ms = C.c_double()
    cnt = C.c_int64()
    _check(ctx, load().dlra_kernel_stats(ctx, C.byref(ms), C.byref(cnt)))
    return ms.value, cnt.value


def kstep_args(grid: dict, r: int, e0: float, de: float, n_sub: int, K0, K1, inv_rho, P, stream=None,
               bk_p=1.77, bk_alpha=0.0022, stage_kernel=0):
    """Argument block of dlra_kstep for torch CUDA float32 tensors K0, K1 (n x r
    column-major, i.e. shape (r, n)), inv_rho (n) and P (nk, r, r) with P_k
    column-major (pass the transposes of the row-major r x r matrices); stage_kernel as
    Solver.set_stage_kernel."""
    a = dlra_kstep_args()
    a.nx, a.ny, a.nz = int(grid["nx"]), int(grid["ny"]), int(grid["nz"])
    a.dx, a.dy, a.dz = float(grid["dx"]), float(grid["dy"]), float(grid["dz"])
    a.r, a.e0, a.de, a.n_sub = int(r), float(e0), float(de), int(n_sub)
    a.bk_p, a.bk_alpha = float(bk_p), float(bk_alpha)
    a.K0, a.K1, a.inv_rho, a.P = K0.data_ptr(), K1.data_ptr(), inv_rho.data_ptr(), P.data_ptr()
    a.cuda_stream = stream
    a.stage_kernel = int(stage_kernel)
    return a


def dlra_kstep(args):
    st = load().dlra_kstep(C.byref(args))
    if st != DLRA_OK:
        raise DlraError(st, load().dlra_last_error(None).decode())


def dlra_kstep_noalloc(args):
    """dlra_kstep on the library's static work space (no device allocation)."""
    st = load().dlra_kstep_noalloc(C.byref(args))
    if st != DLRA_OK:
        raise DlraError(st, load().dlra_last_error(None).decode())


def dlra_stencil_gram(args):
    st = load().dlra_stencil_gram(C.byref(args))
    if st != DLRA_OK:
        raise DlraError(st, load().dlra_last_error(None).decode())


def stencil_gram(grid, spacing, A, B, inv_rho, variant=0):
    """G[k, b, a] = sum_i A[i, a] D_k(rho^-1 B[:, b])[i] for device FP32 tensors A (n x na) and
    B (n x nb), column-major (A[:, a] contiguous: pass A as an (na, n) row-major tensor's
    transpose or as the .T of a contiguous tensor); returns an FP64 device tensor (nk, nb, na)."""
    import torch
    nx, ny, nz = grid
    dx, dy, dz = spacing
    two_d = ny == 1 and dy == 0.0
    nk = 4 if two_d else 6
    n = nx * ny * nz
    assert A.shape[0] == n and B.shape[0] == n and A.stride(0) == 1 and B.stride(0) == 1
    na, nb = A.shape[1], B.shape[1]
    out = torch.empty((nk, nb, na), dtype=torch.float64, device=A.device)
    args = dlra_stencil_gram_args(nx, ny, nz, dx, dy, dz, na, nb, A.data_ptr(), A.stride(1), B.data_ptr(),
                                  B.stride(1), inv_rho.data_ptr(), out.data_ptr(), int(variant),
                                  torch.cuda.current_stream(A.device).cuda_stream)
    dlra_stencil_gram(args)
    return out


def straggling_tables(e_min, e_max, n_elem=128, bk_p=1.77, bk_alpha=0.0022, t100=1.72e-4, straggling=True):
    """Host tables of the straggling ray model (dlra_straggling_tables): mass (3 G,) and the
    block-tridiagonal adv, sipg, rem (G, 3, 3, 3) for G = n_elem energy elements."""
    a = dlra_straggling_args(float(e_min), float(e_max), int(n_elem), float(bk_p), float(bk_alpha), float(t100),
                             int(bool(straggling)))
    mass = np.zeros(3 * n_elem)
    adv = np.zeros((n_elem, 3, 3, 3))
    sipg = np.zeros((n_elem, 3, 3, 3))
    rem = np.zeros((n_elem, 3, 3, 3))
    st = load().dlra_straggling_tables(C.byref(a), _dptr(mass), _dptr(adv), _dptr(sipg), _dptr(rem))
    if st != DLRA_OK:
        raise DlraError(st, load().dlra_last_error(None).decode())
    return mass, adv, sipg, rem


def straggling_trace(cfg, beam, f_cell, tau_cell, n_elem=128, h_max=0.01, straggling=True, stream=None):
    """Uncollided fluence and deposit of one unit-weight beam with energy straggling
    (dlra_straggling_trace) on the grid and energy bins of cfg. f_cell, tau_cell: FP64 device
    tensors (n,), the stopping and removal factors. Returns FP64 device tensors psi (K, n), e_u (n)."""
    import torch
    dev = f_cell.device
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    K = cfg["n_steps"]
    psi = torch.empty((K, n), dtype=torch.float64, device=dev)
    e_u = torch.empty(n, dtype=torch.float64, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    a = dlra_straggling_trace_args(
        cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"], cfg["e_min"], cfg["e_max"], K,
        int(n_elem), float(h_max), cfg["bk_p"], cfg["bk_alpha"], cfg["t100"], int(bool(straggling)),
        float(beam["energy"]), float(beam.get("energy_sigma", 0.0)), float(beam.get("spot_sigma", 0.0)),
        (C.c_double * 3)(*beam["pos"]), (C.c_double * 3)(*beam["dir"]),
        f_cell.data_ptr(), tau_cell.data_ptr(), psi.data_ptr(), e_u.data_ptr(), st)
    code = load().dlra_straggling_trace(C.byref(a))
    if code != DLRA_OK:
        raise DlraError(code, load().dlra_last_error(None).decode())
    return psi, e_u


def dlra_launch_count(ctx) -> int:
    return int(load().dlra_launch_count(ctx))


def dlra_last_error(ctx) -> str:
    return load().dlra_last_error(ctx).decode()


def dlra_destroy(ctx):
    if ctx is not None and ctx.value:
        load().dlra_destroy(ctx)


def _is_cuda_tensor(x):
    try:
        import torch
    except ImportError:
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


class Solver:
    """One context: configuration dict, materials, mixture weights, beams."""

    def __init__(self, cfg: dict, materials=None, w=None, beams=(), stream=None):
        self.cfg = dict(cfg)
        self.n = int(cfg["nx"]) * int(cfg["ny"]) * int(cfg["nz"])
        self.m = (int(cfg["N"]) + 1) ** 2
        self.K = int(cfg["n_steps"])
        self.rank_max = int(cfg.get("rank_max", cfg.get("rank", 5)))
        self.ctx = dlra_init(cfg, stream)
        self.beam_ids = []
        if materials is not None:
            self.set_materials(materials, w)
        for b in beams:
            self.add_beam(b)

    def set_materials(self, materials, w):
        """Set (or replace, same number of materials) the mixture; replacing retraces and rewinds."""
        self.n_mat = len(materials)
        dlra_set_materials(self.ctx, materials, w)

    def set_beam_weight(self, beam_id, weight):
        dlra_set_beam_weight(self.ctx, beam_id, weight)

    def enable_adjoint(self, checkpoint_interval=16):
        dlra_enable_adjoint(self.ctx, checkpoint_interval)

    def set_adjoint_store(self, keep=True):
        """Keep the replayed forward stage inputs for the reverse sweep (more memory, less work)."""
        dlra_set_adjoint_store(self.ctx, keep)

    def backward(self, dL_de, dw_out=None):
        """(dL/dweight per beam, dL/dw per material and cell) of a loss of the dose."""
        return dlra_backward(self.ctx, dL_de, len(self.beam_ids), self.n_mat, self.n, dw_out)

    def add_beam(self, beam):
        self.beam_ids.append(dlra_add_beam(self.ctx, beam))
        return self.beam_ids[-1]

    def step(self, n_steps=1):
        dlra_step(self.ctx, n_steps)

    def run(self):
        step, _ = self.query()
        if self.K - step:
            self.step(self.K - step)
        return self.dose()

    def dose(self, out=None, per_mass=False):
        return dlra_dose(self.ctx, self.n, out, per_mass)

    def query(self):
        return dlra_query(self.ctx, len(self.beam_ids))

    def rank_log(self, beam_id=0):
        return dlra_rank_log(self.ctx, beam_id, self.K)

    def get_state(self, beam_id=0):
        return dlra_get_state(self.ctx, beam_id, self.n, self.m, self.rank_max)

    def set_state(self, X, S, W, beam_id=0):
        dlra_set_state(self.ctx, beam_id, X, S, W, self.rank_max)

    def source(self, k, beam_id=0):
        return dlra_get_source(self.ctx, beam_id, k, self.n)

    def tables(self):
        return dlra_get_tables(self.ctx, self.m)

    def substeps(self):
        return dlra_get_substeps(self.ctx, self.K)

    def reset(self, retrace=True):
        dlra_reset(self.ctx, retrace)

    def set_profiling(self, enable=True):
        dlra_set_profiling(self.ctx, enable)

    def autotune(self):
        """Time the launch variants of the heavy kernels here and keep the fastest."""
        return dlra_autotune(self.ctx)

    def set_stage_kernel(self, variant):
        """0 per-cell FMA, 1 tensor cores (FP32 path), 2 brick-staged FMA, 3 cell pairs (FP32, nx even),
        4 / 5 TMA-staged tensor cores with 128- / 256-cell bricks (FP32, 3-D, nx % 4 == 0, rank capacity >= 32),
        6 the same as one persistent CTA per SM with overlapped epilogue, 7 128-cell bricks with the A operand
        in tensor memory, 8 variant 7 on 2-CTA clusters sharing multicast halo and B copies, 9 variant 7 on
        bricks of three tiles along z sharing one halo box and B image, 10 variant 7 on chunks of eight columns,
        11 variant 7 with eight formation warps, 12 variant 11 staging each chunk as five TMA boxes (brick with
        its x halo, four y/z faces) with an FP32 B image split in shared memory, 13 variant 12 with the B image
        copied already split."""
        dlra_set_stage_kernel(self.ctx, variant)

    def set_stencil_gram_kernel(self, variant):
        """0 FMA, 1 tensor cores (FP32 path), 2 tensor cores with a sliding TMA window (FP32, 3-D; else 1)."""
        dlra_set_stencil_gram_kernel(self.ctx, variant)

    def set_tensor_cores(self, enable=True):
        """Run the streaming stage on the tcgen05 tensor cores (FP32-mixed path)."""
        dlra_set_tensor_cores(self.ctx, enable)

    def set_straggling(self, enable=True, n_elem=128, h_max=0.01, straggling=True):
        """Uncollided source from the energy-DG straggling tracer (Sec. 3.2); re-traces the
        beams already added."""
        dlra_set_straggling(self.ctx, enable, n_elem, h_max, straggling)
        if self.beam_ids:
            self.reset(retrace=True)

    def set_gram_kernel(self, variant):
        """0 FMA, 1 tensor cores for the cell-side tall-skinny Grams (FP32 path, tall), 2 tensor cores always."""
        dlra_set_gram_kernel(self.ctx, variant)

    def set_apply_kernel(self, variant):
        """0 FMA, 1 tensor cores for the cell-side tall-skinny products (FP32 path)."""
        dlra_set_apply_kernel(self.ctx, variant)

    def set_joint(self, enable=True):
        """All beams share one low-rank state (call before the first step)."""
        dlra_set_joint(self.ctx, enable)

    def set_graphs(self, enable=True):
        """Capture each dlra_step call as a CUDA graph and replay it on repeated solves."""
        dlra_set_graphs(self.ctx, enable)

    def kernel_stats(self):
        return dlra_kernel_stats(self.ctx)

    def launch_count(self):
        return dlra_launch_count(self.ctx)

    def close(self):
        dlra_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self.ctx is not None:
                self.close()
        except Exception:
            pass


_DOSE_FN = None


def differentiable_dose(solver: "Solver", materials, w, weights):
    """Dose e (CUDA float64, n) as a differentiable function of the mixture weights
    ``w`` (CUDA float64 tensor (n_mat, n)) and the beam weights ``weights`` (float64
    tensor (n_beams,)). The forward replaces the mixture (which retraces and rewinds
    every beam), sets the beam weights and runs all energy steps; the backward is the
    library's reverse sweep (``solver.enable_adjoint`` must have been called)."""
    global _DOSE_FN
    import torch

    if _DOSE_FN is None:
        class _DoseFunction(torch.autograd.Function):
            @staticmethod
            def forward(fctx, solver_, materials_, w_, weights_):
                solver_.set_materials(materials_, w_.detach().contiguous())
                for b, wt in enumerate(weights_.detach().cpu().tolist()):
                    solver_.set_beam_weight(b, wt)
                solver_.step(solver_.K)
                e = torch.empty(solver_.n, dtype=torch.float64, device=w_.device)
                solver_.dose(out=e)
                fctx.solver = solver_
                fctx.wdev = weights_.device
                return e

            @staticmethod
            def backward(fctx, grad_e):
                sv = fctx.solver
                dw = torch.empty((sv.n_mat, sv.n), dtype=torch.float64, device=grad_e.device)
                dbeta, _ = sv.backward(grad_e.detach().to(torch.float64).contiguous(), dw_out=dw)
                return None, None, dw, torch.as_tensor(dbeta, dtype=torch.float64, device=fctx.wdev)

        _DOSE_FN = _DoseFunction
    return _DOSE_FN.apply(solver, materials, w, weights)
