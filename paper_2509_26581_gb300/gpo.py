"""ctypes binding of libgpo (include/gpo.h): same names as the C ABI, argument
marshalling only.  Every step of the optimiser runs in the library's CUDA kernels;
this module never computes any part of it.

`Graph` is a thin convenience wrapper over the C calls for numpy / torch arrays.
Importing this module loads libgpo.so (building it first if needed) and raises
if the library cannot be loaded; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

GPO_OK = 0
GPO_ERR_ARG, GPO_ERR_OOM, GPO_ERR_STATE, GPO_ERR_NUMERIC = -1, -2, -3, -4
GPO_ERR_CUDA, GPO_ERR_TIMEOUT, GPO_ERR_UNSUPPORTED = -5, -6, -7
GPO_SOLVER_SCHUR, GPO_SOLVER_FULL = 0, 1
GPO_FP64, GPO_FP32, GPO_FP32_BF16 = 0, 1, 2
GPO_V_BA_CAMERA9, GPO_V_POINT3, GPO_V_NAV15 = 0, 1, 2
GPO_E_BA_REPROJ, GPO_E_STEREO, GPO_E_IMU, GPO_E_BIAS_RW, GPO_E_BIAS_PRIOR, GPO_E_MONO = 0, 1, 2, 3, 4, 5
GPO_IMU_MEAS_LEN = 67
GPO_LOSS_NONE, GPO_LOSS_HUBER = 0, 1
PRECISIONS = {"fp64": GPO_FP64, "fp32": GPO_FP32, "bf16": GPO_FP32_BF16}

_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class gpo_graph_desc(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32),
                ("reserve_vertices", C.c_int64), ("reserve_edges", C.c_int64),
                ("cuda_stream", C.c_void_p), ("alloc", _ALLOC), ("free", _FREE),
                ("alloc_ctx", C.c_void_p), ("memory_budget", C.c_size_t),
                ("chunk_edges", C.c_int32), ("spmv_variant", C.c_int32), ("spmv_kernel", C.c_int32),
                ("reserved0", C.c_int32), ("j_bytes", C.c_int64)]


class gpo_lm_params(C.Structure):
    _fields_ = [("initial_damping", C.c_double), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double), ("diag_min", C.c_double), ("diag_max", C.c_double),
                ("damping_mode", C.c_int32), ("pcg_max_iters", C.c_int32),
                ("pcg_tol", C.c_double), ("pcg_tol_relative", C.c_int32),
                ("pcg_rejection_ratio", C.c_double), ("pcg_normalize", C.c_int32),
                ("pcg_restart_every", C.c_int32), ("solver", C.c_int32), ("initial_nu", C.c_double)]


class gpo_report(C.Structure):
    _fields_ = [("initial_cost", C.c_double), ("final_cost", C.c_double),
                ("final_lambda", C.c_double), ("iterations", C.c_int32),
                ("accepted", C.c_int32), ("pcg_iters_total", C.c_int32), ("reserved0", C.c_int32),
                ("final_nu", C.c_double)]


class gpo_iter_record(C.Structure):
    _fields_ = [("cost", C.c_double), ("cand_cost", C.c_double), ("model_decrease", C.c_double),
                ("rho", C.c_double), ("lambda_", C.c_double), ("pcg_residual", C.c_double),
                ("accepted", C.c_int32), ("pcg_iters", C.c_int32), ("pcg_products", C.c_int32),
                ("pcg_failed", C.c_int32)]


class gpo_graph_info_t(C.Structure):
    _fields_ = [("cameras", C.c_int64), ("points", C.c_int64), ("edges", C.c_int64),
                ("extra_edges", C.c_int64), ("chunks", C.c_int64), ("slots", C.c_int64),
                ("chunk_edges", C.c_int32), ("spmv_variant", C.c_int32), ("spmv_kernel", C.c_int32),
                ("reserved0", C.c_int32), ("j_bytes", C.c_int64)]


class gpo_kernel_profile(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("timed_launches", C.c_int64),
                ("active_launches", C.c_int64), ("total_ms", C.c_double), ("active_ms", C.c_double)]


class gpo_server_desc(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("cuda_stream", C.c_void_p),
                ("memory_budget", C.c_size_t), ("max_resident", C.c_int32), ("reserved0", C.c_int32)]


_P = C.c_void_p
_PD = C.POINTER(C.c_double)
_PI64 = C.POINTER(C.c_int64)
_SIGS = {
    "gpo_graph_desc_default": (C.c_int, [C.POINTER(gpo_graph_desc)]),
    "gpo_lm_params_default": (C.c_int, [C.POINTER(gpo_lm_params)]),
    "gpo_graph_create": (C.c_int, [C.POINTER(gpo_graph_desc), C.POINTER(_P)]),
    "gpo_graph_destroy": (C.c_int, [_P]),
    "gpo_add_vertices": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int64, _PI64]),
    "gpo_add_edges": (C.c_int, [_P, C.c_int32, C.c_int64, _P, _P, _P, C.c_int32, C.c_double, _PI64]),
    "gpo_set_fixed": (C.c_int, [_P, C.c_int64, C.c_int32]),
    "gpo_set_edge_active": (C.c_int, [_P, C.c_int64, C.c_int32]),
    "gpo_set_initial": (C.c_int, [_P, C.c_int64, C.c_int64, _P, C.c_int32]),
    "gpo_optimize": (C.c_int, [_P, C.c_int32, C.POINTER(gpo_lm_params), C.POINTER(gpo_report)]),
    "gpo_get_cost": (C.c_int, [_P, _PD]),
    "gpo_get_state": (C.c_int, [_P, C.c_int64, C.c_int64, _P, C.c_int32]),
    "gpo_get_history": (C.c_int, [_P, C.POINTER(gpo_iter_record), C.c_int32, C.POINTER(C.c_int32)]),
    "gpo_memory_footprint": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "gpo_graph_plan": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "gpo_graph_info": (C.c_int, [_P, C.POINTER(gpo_graph_info_t)]),
    "gpo_set_profiling": (C.c_int, [_P, C.c_int32]),
    "gpo_get_profile": (C.c_int, [_P, C.POINTER(gpo_kernel_profile), C.c_int32, C.POINTER(C.c_int32)]),
    "gpo_last_error": (C.c_char_p, [_P]),
    "gpo_version": (C.c_char_p, []),
    "gpo_optimize_batch": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int32, C.POINTER(gpo_lm_params),
                                     C.POINTER(gpo_report)]),
    "gpo_server_desc_default": (C.c_int, [C.POINTER(gpo_server_desc)]),
    "gpo_server_create": (C.c_int, [C.POINTER(gpo_server_desc), C.POINTER(_P)]),
    "gpo_server_destroy": (C.c_int, [_P]),
    "gpo_server_submit": (C.c_int, [_P, _P, C.c_int32, C.POINTER(gpo_lm_params), _PI64]),
    "gpo_server_step": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "gpo_server_poll": (C.c_int, [_P, C.c_int64, C.POINTER(C.c_int32), C.POINTER(gpo_report)]),
    "gpo_server_memory": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "gpo_server_last_error": (C.c_char_p, [_P]),
    "gpo_ba_cost_noalloc": (C.c_int, [C.c_int32, _P, _P, _P, _P, _P, _P, C.c_int64, C.c_double, _P]),
    "gpo_set_stereo_camera": (C.c_int, [_P, _P]),
    "gpo_set_fisheye": (C.c_int, [_P, _P]),
    "gpo_imu_preintegrate": (C.c_int, [_P, _P, C.c_int64, C.c_double, _P, _P, C.c_double, C.c_double,
                                       _P, _P, _P]),
    "gpo_debug_linearize": (C.c_int, [_P, _P, _P]),
    "gpo_debug_linearize_edges": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "gpo_debug_step": (C.c_int, [_P, C.c_double, C.POINTER(gpo_lm_params), _P, C.POINTER(C.c_int32)]),
    "gpo_debug_schur": (C.c_int, [_P, C.c_double, C.POINTER(gpo_lm_params), _P, _P]),
    "gpo_debug_wait_timeout": (C.c_int, [_P]),
    "gpo_debug_autodiff_edges": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "gpo_fp64_fma_probe": (C.c_int, [_P, C.c_int32, C.c_int32, _P]),
    "gpo_generic_create": (C.c_int, [C.c_int32, C.c_int64, _P, C.c_int32, _P, C.POINTER(_P)]),
    "gpo_generic_destroy": (C.c_int, [_P]),
    "gpo_generic_add_edges": (C.c_int, [_P, C.c_int32, C.c_int64, _P, _P, C.c_int32, C.c_double, _PI64]),
    "gpo_generic_set_fixed": (C.c_int, [_P, C.c_int64, C.c_int32]),
    "gpo_generic_set_edge_active": (C.c_int, [_P, C.c_int64, C.c_int32]),
    "gpo_generic_optimize": (C.c_int, [_P, C.c_int32, C.POINTER(gpo_lm_params), C.POINTER(gpo_report)]),
    "gpo_generic_get_state": (C.c_int, [_P, _P]),
}


def load_library(path: str | None = None) -> C.CDLL:
    path = path or os.environ.get("GPO_LIBRARY") or _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load_library()


class GpoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gpo status {status}: {msg}")
        self.status = status


def _check(st: int, g=None):
    if st != GPO_OK:
        msg = lib.gpo_last_error(g)
        raise GpoError(st, msg.decode() if msg else "")


def default_params(**kw) -> gpo_lm_params:
    p = gpo_lm_params()
    _check(lib.gpo_lm_params_default(C.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Graph:
    """Owns one gpo_graph handle."""

    def __init__(self, precision="fp64", device: int = 0, stream=None, memory_budget: int = 0,
                 reserve_vertices: int = 0, reserve_edges: int = 0, chunk_edges: int = 0,
                 spmv_variant: int = 0):
        d = gpo_graph_desc()
        _check(lib.gpo_graph_desc_default(C.byref(d)))
        d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        d.device = device
        d.cuda_stream = stream
        d.memory_budget = memory_budget
        d.reserve_vertices = reserve_vertices
        d.reserve_edges = reserve_edges
        d.chunk_edges = chunk_edges
        d.spmv_variant = spmv_variant
        self.knobs = dict(chunk_edges=chunk_edges, spmv_variant=spmv_variant)
        h = C.c_void_p()
        _check(lib.gpo_graph_create(C.byref(d), C.byref(h)))
        self.h = h
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            lib.gpo_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def add_vertices(self, kind: int, block_size: int, n: int) -> int:
        first = C.c_int64()
        _check(lib.gpo_add_vertices(self.h, kind, block_size, n, C.byref(first)), self.h)
        return first.value

    def add_edges(self, kind: int, vertex_ids: np.ndarray, meas, info=None,
                  loss_kind: int = GPO_LOSS_NONE, loss_delta: float = 0.0) -> int:
        ids = np.ascontiguousarray(vertex_ids, dtype=np.int64)
        m = None if meas is None else np.ascontiguousarray(meas, dtype=np.float64)
        inf = None if info is None else np.ascontiguousarray(info, dtype=np.float64)
        first = C.c_int64()
        _check(lib.gpo_add_edges(self.h, kind, ids.shape[0], _ptr(ids), None if m is None else _ptr(m),
                                 None if inf is None else _ptr(inf), loss_kind, loss_delta,
                                 C.byref(first)), self.h)
        return first.value

    def set_stereo_camera(self, rig) -> None:
        """rig = [fx fy cx cy baseline, R_cb (9, row-major), t_cb (3)]."""
        a = np.ascontiguousarray(rig, dtype=np.float64).reshape(-1)
        if a.shape[0] != 17:
            raise ValueError("the stereo rig has 17 values")
        _check(lib.gpo_set_stereo_camera(self.h, _ptr(a)), self.h)

    def set_fisheye(self, k) -> None:
        """Kannala-Brandt coefficients [k1 k2 k3 k4] for both cameras of the rig
        (gpo_set_fisheye; after set_stereo_camera)."""
        a = np.ascontiguousarray(k, dtype=np.float64).reshape(-1)
        if a.shape[0] != 4:
            raise ValueError("four fisheye coefficients")
        _check(lib.gpo_set_fisheye(self.h, _ptr(a)), self.h)

    def set_fixed(self, vid: int, fixed: bool = True):
        _check(lib.gpo_set_fixed(self.h, vid, int(fixed)), self.h)

    def set_edge_active(self, eid: int, active: bool):
        _check(lib.gpo_set_edge_active(self.h, eid, int(active)), self.h)

    def set_initial(self, first: int, state) -> None:
        """state: numpy array (host) or torch CUDA tensor (device), float64 rows."""
        if hasattr(state, "data_ptr"):
            n = state.shape[0]
            _check(lib.gpo_set_initial(self.h, first, n, C.c_void_p(state.data_ptr()), 1), self.h)
        else:
            a = np.ascontiguousarray(state, dtype=np.float64)
            _check(lib.gpo_set_initial(self.h, first, a.shape[0], _ptr(a), 0), self.h)

    def get_state(self, first: int, n: int, width: int, out=None):
        """Copies n states out: into `out` when given (a CUDA tensor: device copy; a CPU
        tensor or a C-contiguous float64 numpy array of n x width: host copy, fastest
        from pinned memory), else into a new numpy array."""
        if out is not None and hasattr(out, "data_ptr"):
            on_dev = 1 if getattr(out, "is_cuda", True) else 0
            _check(lib.gpo_get_state(self.h, first, n, C.c_void_p(out.data_ptr()), on_dev), self.h)
            return out
        if out is not None:
            if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != n * width:
                raise ValueError("out must be a C-contiguous float64 array of n x width")
            _check(lib.gpo_get_state(self.h, first, n, _ptr(out), 0), self.h)
            return out
        a = np.empty((n, width), dtype=np.float64)
        _check(lib.gpo_get_state(self.h, first, n, _ptr(a), 0), self.h)
        return a

    def optimize(self, max_iters: int, params: gpo_lm_params | None = None) -> gpo_report:
        rep = gpo_report()
        _check(lib.gpo_optimize(self.h, max_iters, None if params is None else C.byref(params),
                                C.byref(rep)), self.h)
        return rep

    def cost(self) -> float:
        v = C.c_double()
        _check(lib.gpo_get_cost(self.h, C.byref(v)), self.h)
        return v.value

    def history(self, cap: int = 4096) -> list[dict]:
        buf = (gpo_iter_record * cap)()
        n = C.c_int32()
        _check(lib.gpo_get_history(self.h, buf, cap, C.byref(n)), self.h)
        return [dict(cost=r.cost, cand_cost=r.cand_cost, model_decrease=r.model_decrease,
                     rho=r.rho, lam=r.lambda_, pcg_residual=r.pcg_residual,
                     accepted=bool(r.accepted), pcg_iters=r.pcg_iters, pcg_products=r.pcg_products,
                     pcg_failed=r.pcg_failed == 1, pcg_breakdown=r.pcg_failed == 2)
                for r in buf[:n.value]]

    def set_profiling(self, on: bool = True):
        _check(lib.gpo_set_profiling(self.h, int(on)), self.h)

    def profile(self) -> dict:
        buf = (gpo_kernel_profile * 32)()
        n = C.c_int32()
        _check(lib.gpo_get_profile(self.h, buf, 32, C.byref(n)), self.h)
        return {r.name.decode(): dict(launches=r.launches, timed=r.timed_launches,
                                      active=r.active_launches, total_ms=r.total_ms,
                                      active_ms=r.active_ms) for r in buf[:n.value]}

    def info(self) -> dict:
        """Sizes of the finalized graph (gpo_graph_info)."""
        v = gpo_graph_info_t()
        _check(lib.gpo_graph_info(self.h, C.byref(v)), self.h)
        return {k: getattr(v, k) for k, _ in gpo_graph_info_t._fields_}

    def plan(self) -> int:
        """Host-side planning (gpo_graph_plan); returns the planned device bytes."""
        v = C.c_size_t()
        _check(lib.gpo_graph_plan(self.h, C.byref(v)), self.h)
        return v.value

    def footprint(self) -> int:
        v = C.c_size_t()
        _check(lib.gpo_memory_footprint(self.h, C.byref(v)), self.h)
        return v.value

    # diagnostics -----------------------------------------------------------
    def debug_linearize(self, n_edges: int, nav: bool = False):
        """Per edge id: whitened residual rows and Jacobian rows ((2, 12) for BA graphs,
        (9, 30) for graphs of navigation states; see gpo_debug_linearize)."""
        R, K = (9, 30) if nav else (2, 12)
        r = np.zeros((n_edges, R))
        J = np.zeros((n_edges, R, K))
        _check(lib.gpo_debug_linearize(self.h, _ptr(r), _ptr(J)), self.h)
        return r, J

    def debug_linearize_edges(self, edge_ids, nav: bool = False):
        """Rows of the given edges only (gpo_debug_linearize_edges)."""
        ids = np.ascontiguousarray(edge_ids, dtype=np.int64)
        R, K = (9, 30) if nav else (2, 12)
        r = np.zeros((len(ids), R))
        J = np.zeros((len(ids), R, K))
        _check(lib.gpo_debug_linearize_edges(self.h, _ptr(ids), len(ids), _ptr(r), _ptr(J)), self.h)
        return r, J

    def debug_autodiff_edges(self, edge_ids, nav: bool = False):
        """Rows of the given edges by forward-mode automatic differentiation, FP64
        (gpo_debug_autodiff_edges; layout of debug_linearize_edges)."""
        ids = np.ascontiguousarray(edge_ids, dtype=np.int64)
        R, K = (9, 30) if nav else (2, 12)
        r = np.zeros((len(ids), R))
        J = np.zeros((len(ids), R, K))
        _check(lib.gpo_debug_autodiff_edges(self.h, _ptr(ids), len(ids), _ptr(r), _ptr(J)), self.h)
        return r, J

    def debug_step(self, lam: float, n_dof: int, params: gpo_lm_params | None = None):
        dx = np.zeros(n_dof)
        it = C.c_int32()
        _check(lib.gpo_debug_step(self.h, lam, None if params is None else C.byref(params),
                                  _ptr(dx), C.byref(it)), self.h)
        return dx, it.value

    def debug_wait_timeout(self) -> int:
        """gpo_debug_wait_timeout: the status it returns (GPO_ERR_TIMEOUT expected)."""
        return int(lib.gpo_debug_wait_timeout(self.h))

    def debug_schur(self, lam: float, n_cams: int, params: gpo_lm_params | None = None, db: int = 9):
        S = np.zeros((n_cams, db, db))
        g = np.zeros((n_cams, db))
        _check(lib.gpo_debug_schur(self.h, lam, None if params is None else C.byref(params),
                                   _ptr(S), _ptr(g)), self.h)
        return S, g


def optimize_batch(graphs: list, max_iters: int, params: gpo_lm_params | None = None) -> list:
    """Solves the graphs together (one launch per phase for all of them)."""
    n = len(graphs)
    arr = (_P * n)(*[g.h for g in graphs])
    reps = (gpo_report * n)()
    st = lib.gpo_optimize_batch(arr, n, max_iters, None if params is None else C.byref(params), reps)
    _check(st, graphs[0].h)
    return list(reps)


def fp64_fma_probe(stream, n_ctas: int, iters: int, out) -> None:
    """gpo_fp64_fma_probe: queues the FP64 FMA throughput kernel on `stream` (a CUDA
    stream handle or 0) writing n_ctas * 256 doubles to the device tensor `out`; one
    launch performs n_ctas * 256 * iters * 32 FMAs."""
    _check(lib.gpo_fp64_fma_probe(stream, n_ctas, iters, out.data_ptr()))


GPO_GE_CIRCLE, GPO_GE_DISTANCE = 0, 1


class Generic:
    """A graph of 2-dim vertices with edges of the library's generic kinds
    (gpo_generic_*: residuals differentiated in forward mode)."""

    def __init__(self, x0, device: int = 0, stream=None):
        x = np.ascontiguousarray(x0, dtype=np.float64)
        self.n, self.dim = x.shape
        h = _P()
        _check(lib.gpo_generic_create(self.dim, self.n, _ptr(x), device, stream, C.byref(h)))
        self.h = h

    def add_edges(self, kind: int, vertex_ids, meas, loss_kind: int = GPO_LOSS_NONE, loss_delta: float = 0.0) -> int:
        ids = np.ascontiguousarray(vertex_ids, dtype=np.int64)
        m = np.ascontiguousarray(meas, dtype=np.float64)
        first = C.c_int64()
        _check(lib.gpo_generic_add_edges(self.h, kind, ids.shape[0], _ptr(ids), _ptr(m), loss_kind, loss_delta,
                                         C.byref(first)))
        return first.value

    def set_fixed(self, vid: int, fixed: bool = True):
        _check(lib.gpo_generic_set_fixed(self.h, vid, int(fixed)))

    def set_edge_active(self, eid: int, active: bool):
        _check(lib.gpo_generic_set_edge_active(self.h, eid, int(active)))

    def optimize(self, max_iters: int, params: gpo_lm_params | None = None) -> gpo_report:
        rep = gpo_report()
        _check(lib.gpo_generic_optimize(self.h, max_iters, None if params is None else C.byref(params),
                                        C.byref(rep)))
        return rep

    def state(self) -> np.ndarray:
        out = np.empty((self.n, self.dim))
        _check(lib.gpo_generic_get_state(self.h, _ptr(out)))
        return out

    def close(self):
        if self.h:
            lib.gpo_generic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop over the C ABI (gpo_server_*)."""

    def __init__(self, precision="bf16", device: int = 0, stream=None, memory_budget: int = 0,
                 max_resident: int = 1024):
        d = gpo_server_desc()
        _check(lib.gpo_server_desc_default(C.byref(d)))
        d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        d.device = device
        d.cuda_stream = stream
        d.memory_budget = memory_budget
        d.max_resident = max_resident
        h = C.c_void_p()
        _check(lib.gpo_server_create(C.byref(d), C.byref(h)))
        self.h = h
        self.graphs = {}

    def _check(self, st):
        if st != GPO_OK:
            msg = lib.gpo_server_last_error(self.h)
            raise GpoError(st, msg.decode() if msg else "")

    def submit(self, graph: "Graph", max_iters: int, params: gpo_lm_params | None = None) -> int:
        t = C.c_int64()
        self._check(lib.gpo_server_submit(self.h, graph.h, max_iters,
                                          None if params is None else C.byref(params), C.byref(t)))
        self.graphs[t.value] = graph
        return t.value

    def step(self) -> tuple[int, int, int]:
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(lib.gpo_server_step(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def poll(self, ticket: int):
        done = C.c_int32()
        rep = gpo_report()
        self._check(lib.gpo_server_poll(self.h, ticket, C.byref(done), C.byref(rep)))
        return rep if done.value else None

    def memory(self) -> int:
        v = C.c_size_t()
        self._check(lib.gpo_server_memory(self.h, C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None):
            lib.gpo_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def _tuned(kw: dict, n_edges: int, precision, model: str) -> dict:
    """Adds the autotuned schedule knobs (chunk size, Schur-product kernel) for this size
    class unless the caller set either of them."""
    if "chunk_edges" in kw or "spmv_variant" in kw:
        return kw
    from . import autotune
    name = precision if isinstance(precision, str) else {v: k for k, v in PRECISIONS.items()}[int(precision)]
    return {**autotune.choose(int(n_edges), name, model), **kw}


def ba_graph(cams, pts, cam_idx, pt_idx, obs, huber_delta=None, precision="fp64",
             cam_fixed=None, pt_fixed=None, active=None, info=None, **kw) -> tuple[Graph, int, int]:
    """Builds a BA graph: cameras get ids [0, C), points [C, C + P).  Returns
    (graph, first camera id, first point id)."""
    kw = _tuned(kw, len(cam_idx), precision, "ba")
    g = Graph(precision, **kw)
    C_ = cams.shape[0]
    P_ = pts.shape[0]
    c0 = g.add_vertices(GPO_V_BA_CAMERA9, 9, C_)
    p0 = g.add_vertices(GPO_V_POINT3, 3, P_)
    ids = np.stack([np.asarray(cam_idx, np.int64) + c0, np.asarray(pt_idx, np.int64) + p0], axis=1)
    if huber_delta is None:
        g.add_edges(GPO_E_BA_REPROJ, ids, obs, info)
    else:
        g.add_edges(GPO_E_BA_REPROJ, ids, obs, info, GPO_LOSS_HUBER, float(huber_delta))
    g.set_initial(c0, cams)
    g.set_initial(p0, pts)
    if cam_fixed is not None:
        for c in np.nonzero(cam_fixed)[0]:
            g.set_fixed(c0 + int(c))
    if pt_fixed is not None:
        for p in np.nonzero(pt_fixed)[0]:
            g.set_fixed(p0 + int(p))
    if active is not None:
        for e in np.nonzero(~np.asarray(active, bool))[0]:
            g.set_edge_active(int(e), False)
    return g, c0, p0


def imu_preintegrate(gyro, acc, dt: float, bg0, ba0, sigma_g: float, sigma_a: float, with_info: bool = True):
    """Library preintegration of one keyframe interval (gpo_imu_preintegrate).
    Returns (record of GPO_IMU_MEAS_LEN doubles, covariance 9x9, information 9x9 or None)."""
    w = np.ascontiguousarray(gyro, dtype=np.float64).reshape(-1, 3)
    a = np.ascontiguousarray(acc, dtype=np.float64).reshape(-1, 3)
    if w.shape != a.shape:
        raise ValueError("gyro and acc must have the same number of samples")
    b_g = np.ascontiguousarray(bg0, dtype=np.float64).reshape(3)
    b_a = np.ascontiguousarray(ba0, dtype=np.float64).reshape(3)
    meas = np.zeros(GPO_IMU_MEAS_LEN)
    cov = np.zeros((9, 9))
    info = np.zeros((9, 9))
    _check(lib.gpo_imu_preintegrate(_ptr(w), _ptr(a), w.shape[0], float(dt), _ptr(b_g), _ptr(b_a),
                                    float(sigma_g), float(sigma_a), _ptr(meas), _ptr(cov),
                                    _ptr(info) if with_info else None))
    return meas, cov, (info if with_info else None)


def stereo_rig(camera: dict) -> np.ndarray:
    """[fx fy cx cy baseline, R_cb, t_cb] of a camera description."""
    return np.r_[camera["fx"], camera["fy"], camera["cx"], camera["cy"], camera["baseline"],
                 np.asarray(camera["R_cb"], float).reshape(9), np.asarray(camera["t_cb"], float).reshape(3)]


def vi_graph(p, nav=None, pts=None, precision="fp64", prior_sigma=(1e-2, 1e-1), huber=True, imu=None,
             imu_huber=None, mono=None, **kw):
    """Builds the visual-inertial graph of a VIProblem-like record: navigation states get
    ids [0, K), landmarks [K, K + P); edges in this order: stereo (Huber), inertial between
    consecutive keyframes (preintegrated by the library at the initial biases of the first
    keyframe of each pair), bias random walk (information diag 1 / (sigma^2 T)), and a
    zero bias prior on keyframe 0 (information diag 1 / prior_sigma^2).  imu = (records
    (K-1, GPO_IMU_MEAS_LEN), information (K-1, 9, 9)) supplies the inertial edges instead;
    imu_huber puts a Huber loss of that threshold on them; mono (a boolean mask over the
    observations) adds the masked ones as monocular left-camera edges, after the stereo
    ones.  Returns (graph, first navigation id, first landmark id, edge-id ranges by kind)."""
    nav = p.nav0 if nav is None else nav
    pts = p.pts0 if pts is None else pts
    kw = _tuned(kw, len(p.kf_idx), precision, "vi")
    g = Graph(precision, **kw)
    K, P = nav.shape[0], pts.shape[0]
    n0 = g.add_vertices(GPO_V_NAV15, 15, K)
    p0 = g.add_vertices(GPO_V_POINT3, 3, P)
    g.set_stereo_camera(stereo_rig(p.camera))
    if p.camera.get("fisheye") is not None:   # Kannala-Brandt coefficients of the rig
        g.set_fisheye(p.camera["fisheye"])
    ids = np.stack([np.asarray(p.kf_idx, np.int64) + n0, np.asarray(p.pt_idx, np.int64) + p0], axis=1)
    ranges = {}
    keep = np.ones(ids.shape[0], bool) if mono is None else ~np.asarray(mono, bool)
    lk, ld = (GPO_LOSS_HUBER, float(p.huber_delta)) if huber else (GPO_LOSS_NONE, 0.0)
    obs = np.asarray(p.obs, np.float64)
    e0 = g.add_edges(GPO_E_STEREO, ids[keep], obs[keep], None, lk, ld)
    ranges["stereo"] = (e0, e0 + int(keep.sum()))
    if not keep.all():   # monocular edges: the left camera's two pixels
        e0 = g.add_edges(GPO_E_MONO, ids[~keep], obs[~keep, :2], None, lk, ld)
        ranges["mono"] = (e0, e0 + int((~keep).sum()))
    if K > 1:
        if imu is not None:
            meas, info = (np.asarray(a, np.float64) for a in imu)
        else:
            meas = np.zeros((K - 1, GPO_IMU_MEAS_LEN))
            info = np.zeros((K - 1, 9, 9))
            for k in range(K - 1):
                meas[k], _, info[k] = imu_preintegrate(p.imu_gyro[k], p.imu_acc[k], p.dt, nav[k, 10:13],
                                                       nav[k, 13:16], p.noise["sigma_g"], p.noise["sigma_a"])
        ij = np.stack([np.arange(K - 1), np.arange(1, K)], axis=1).astype(np.int64) + n0
        if imu_huber is None:
            e0 = g.add_edges(GPO_E_IMU, ij, meas, info)
        else:   # Huber on the inertial edges' whitened residual
            e0 = g.add_edges(GPO_E_IMU, ij, meas, info, GPO_LOSS_HUBER, float(imu_huber))
        ranges["imu"] = (e0, e0 + K - 1)
        T = meas[:, 60]
        w2 = np.concatenate([np.tile((1.0 / (p.noise["sigma_bg"] ** 2 * T))[:, None], (1, 3)),
                             np.tile((1.0 / (p.noise["sigma_ba"] ** 2 * T))[:, None], (1, 3))], axis=1)
        e0 = g.add_edges(GPO_E_BIAS_RW, ij, None, np.stack([np.diag(x) for x in w2]))
        ranges["bias_rw"] = (e0, e0 + K - 1)
    pw = np.diag(np.r_[np.full(3, prior_sigma[0] ** -2.0), np.full(3, prior_sigma[1] ** -2.0)])
    e0 = g.add_edges(GPO_E_BIAS_PRIOR, np.array([[n0]], np.int64), np.zeros((1, 6)), pw[None])
    ranges["bias_prior"] = (e0, e0 + 1)
    g.set_initial(n0, nav)
    g.set_initial(p0, pts)
    return g, n0, p0, ranges
