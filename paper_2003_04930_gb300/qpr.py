"""Thin Python binding of the C ABI in ``include/qpr.h`` (ctypes).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libqpr.so``. Density matrices may be torch complex128 CUDA tensors
(passed by device pointer) or NumPy complex128 arrays (host memory; the
library copies them in and out). There is no CPU fallback: if the library
cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqpr.so")

QPR_OK, QPR_E_ARG, QPR_E_GRAPH, QPR_E_CUDA, QPR_E_OOM, QPR_E_UNSTABLE, QPR_E_NOT_CONVERGED, \
    QPR_E_TIMEOUT, QPR_E_NONFINITE = range(9)
QPR_FP64, QPR_MIXED = 0, 1
QPR_HDIAG_ZERO, QPR_HDIAG_NEG_OUTDEG = 0, 1
QPR_DANGLING_F, QPR_DANGLING_UNIFORM = 0, 1
QPR_BACKEND_AUTO, QPR_BACKEND_DENSE, QPR_BACKEND_SPARSE = 0, 1, 2
(QPR_SPARSE_FORM_AUTO, QPR_SPARSE_FORM_COLUMNS, QPR_SPARSE_FORM_TILES, QPR_SPARSE_FORM_COLUMNS_PERSISTENT,
 QPR_SPARSE_FORM_COLUMNS_GATHER) = 0, 1, 2, 3, 5

# every entry point declared in include/qpr.h
EXPORTED = (
    "qpr_default_options", "qpr_create", "qpr_destroy", "qpr_last_error", "qpr_status_string",
    "qpr_n", "qpr_backend", "qpr_sparse_form", "qpr_sparse_plan", "qpr_h_spread", "qpr_max_stable_dt", "qpr_rhs", "qpr_residual", "qpr_evolve",
    "qpr_steady_state", "qpr_populations", "qpr_profile_step", "qpr_profile_chain", "qpr_rhs_noalloc", "qpr_batch_steady_state",
    "qpr_gnn_param_count", "qpr_gnn_create", "qpr_gnn_destroy", "qpr_gnn_get_params", "qpr_gnn_set_params",
    "qpr_gnn_predict", "qpr_gnn_loss_grad", "qpr_gnn_train", "qpr_autotune", "qpr_pagerank", "qpr_hub_classes",
    "qpr_rkf45",
)
QPR_NOALLOC_MAX_N = 256


class qpr_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("h_diag", ctypes.c_int32), ("dangling", ctypes.c_int32),
                ("graph_steps", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("backend", ctypes.c_int32),
                ("ref_refresh", ctypes.c_int32), ("sparse_form", ctypes.c_int32),
                ("test_fault", ctypes.c_int32), ("row_splits", ctypes.c_int32),
                ("adaptive_refresh", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class qpr_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("substeps_m", ctypes.c_int64), ("t", ctypes.c_double),
                ("residual", ctypes.c_double), ("trace_before", ctypes.c_double),
                ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("converged", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k in
                ("steps", "substeps_m", "t", "residual", "trace_before", "seconds", "kernel_launches",
                 "converged")}


class qpr_profile(ctypes.Structure):
    _fields_ = [("product_ms", ctypes.c_double), ("epilogue_ms", ctypes.c_double), ("gain_ms", ctypes.c_double),
                ("refresh_ms", ctypes.c_double), ("step_ms", ctypes.c_double),
                ("launches_per_step", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k in
                ("product_ms", "epilogue_ms", "gain_ms", "refresh_ms", "step_ms", "launches_per_step")}


class qpr_rkf45_options(ctypes.Structure):
    _fields_ = [("h0", ctypes.c_double), ("step_tol", ctypes.c_double), ("h_max", ctypes.c_double),
                ("t_end", ctypes.c_double), ("order", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class qpr_rkf45_stats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int64), ("rejected", ctypes.c_int64), ("t", ctypes.c_double),
                ("h_next", ctypes.c_double), ("residual", ctypes.c_double), ("last_discrepancy", ctypes.c_double),
                ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_int64), ("converged", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k in
                ("accepted", "rejected", "t", "h_next", "residual", "last_discrepancy", "seconds",
                 "kernel_launches", "converged")}


class qpr_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("omega", ctypes.c_double), ("rho", ctypes.c_void_p)]


class qpr_gnn_sample(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("omega", ctypes.c_double), ("p", ctypes.c_void_p)]


class qpr_tune_result(ctypes.Structure):
    _fields_ = [("backend", ctypes.c_int32), ("ref_refresh", ctypes.c_int32), ("ms_per_step", ctypes.c_double),
                ("from_cache", ctypes.c_int32), ("sparse_form", ctypes.c_int32), ("row_splits", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 1)]


class QprError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libqpr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i64, f64, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    lib.qpr_default_options.argtypes = [ctypes.POINTER(qpr_options)]
    lib.qpr_default_options.restype = st
    lib.qpr_create.argtypes = [ctypes.POINTER(vp), i64, i64, vp, vp, vp, f64, f64, ctypes.POINTER(qpr_options)]
    lib.qpr_create.restype = st
    lib.qpr_destroy.argtypes = [vp]
    lib.qpr_destroy.restype = None
    lib.qpr_last_error.argtypes = [vp]
    lib.qpr_last_error.restype = ctypes.c_char_p
    lib.qpr_status_string.argtypes = [st]
    lib.qpr_status_string.restype = ctypes.c_char_p
    lib.qpr_n.argtypes = [vp]
    lib.qpr_n.restype = i64
    lib.qpr_backend.argtypes = [vp]
    lib.qpr_backend.restype = ctypes.c_int32
    lib.qpr_sparse_form.argtypes = [vp]
    lib.qpr_sparse_form.restype = ctypes.c_int32
    lib.qpr_sparse_plan.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.qpr_sparse_plan.restype = st
    lib.qpr_h_spread.argtypes = [vp]
    lib.qpr_h_spread.restype = f64
    lib.qpr_max_stable_dt.argtypes = [vp]
    lib.qpr_max_stable_dt.restype = f64
    lib.qpr_rhs.argtypes = [vp, vp, vp]
    lib.qpr_rhs.restype = st
    lib.qpr_residual.argtypes = [vp, vp, ctypes.POINTER(f64)]
    lib.qpr_residual.restype = st
    lib.qpr_evolve.argtypes = [vp, vp, f64, i64]
    lib.qpr_evolve.restype = st
    lib.qpr_steady_state.argtypes = [vp, vp, f64, f64, i64, ctypes.POINTER(qpr_stats)]
    lib.qpr_steady_state.restype = st
    lib.qpr_profile_step.argtypes = [vp, vp, f64, i64, ctypes.POINTER(qpr_profile)]
    lib.qpr_profile_step.restype = st
    lib.qpr_profile_chain.argtypes = [vp, vp, f64, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    lib.qpr_profile_chain.restype = st
    lib.qpr_rhs_noalloc.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, f64, f64, ctypes.c_int32, vp, vp, vp]
    lib.qpr_rhs_noalloc.restype = st
    lib.qpr_batch_steady_state.argtypes = [i64, ctypes.POINTER(qpr_problem), f64, f64, f64, i64,
                                           ctypes.POINTER(qpr_options), ctypes.POINTER(qpr_stats)]
    lib.qpr_batch_steady_state.restype = st
    lib.qpr_gnn_param_count.argtypes = []
    lib.qpr_gnn_param_count.restype = i64
    lib.qpr_gnn_create.argtypes = [ctypes.POINTER(vp), ctypes.c_uint64, ctypes.c_int32]
    lib.qpr_gnn_create.restype = st
    lib.qpr_gnn_destroy.argtypes = [vp]
    lib.qpr_gnn_destroy.restype = None
    lib.qpr_gnn_get_params.argtypes = [vp, vp]
    lib.qpr_gnn_get_params.restype = st
    lib.qpr_gnn_set_params.argtypes = [vp, vp]
    lib.qpr_gnn_set_params.restype = st
    lib.qpr_gnn_predict.argtypes = [vp, i64, i64, vp, vp, vp, f64, f64, vp]
    lib.qpr_gnn_predict.restype = st
    lib.qpr_gnn_loss_grad.argtypes = [vp, ctypes.POINTER(qpr_gnn_sample), f64, ctypes.POINTER(f64), vp]
    lib.qpr_gnn_loss_grad.restype = st
    lib.qpr_gnn_train.argtypes = [vp, i64, ctypes.POINTER(qpr_gnn_sample), f64, ctypes.c_int32, ctypes.c_int32, f64,
                                  ctypes.c_uint64, vp]
    lib.qpr_gnn_train.restype = st
    lib.qpr_autotune.argtypes = [i64, i64, vp, vp, vp, f64, f64, f64, ctypes.POINTER(qpr_options), ctypes.c_char_p,
                                 ctypes.POINTER(qpr_tune_result)]
    lib.qpr_autotune.restype = st
    lib.qpr_populations.argtypes = [vp, vp, vp, vp]
    lib.qpr_populations.restype = st
    lib.qpr_rkf45.argtypes = [vp, vp, ctypes.POINTER(qpr_rkf45_options), f64, i64, ctypes.POINTER(qpr_rkf45_stats)]
    lib.qpr_rkf45.restype = st
    lib.qpr_pagerank.argtypes = [vp, f64, i64, vp, ctypes.POINTER(i64)]
    lib.qpr_pagerank.restype = st
    lib.qpr_hub_classes.argtypes = [vp, vp, f64, vp, vp]
    lib.qpr_hub_classes.restype = st
    _lib = lib
    return lib


def status_name(status: int) -> str:
    try:
        return load_library().qpr_status_string(int(status)).decode()
    except ImportError:
        return f"status {status}"


def _ptr(x):
    """Raw pointer of a torch tensor (device or host) or a NumPy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check_rho(rho, n):
    dt = getattr(rho, "dtype", None)
    ok = (str(dt) in ("torch.complex128", "complex128"))
    if not ok or tuple(rho.shape) != (n, n):
        raise ValueError(f"rho must be a contiguous ({n}, {n}) complex128 array or tensor")


class Solver:
    """One problem (graph, alpha, omega) bound to a CUDA device.

    The keyword options are the fields of qpr_options (include/qpr.h):
    precision (QPR_FP64 or QPR_MIXED), backend, h_diag, dangling,
    graph_steps, ref_refresh, sparse_form (the mixed sparse stage's form),
    row_splits (COLUMNS, COLUMNS_GATHER), adaptive_refresh (steady-state
    solves of the mixed form) and test_fault (testing only); stream is a
    torch stream (or a raw cudaStream_t) the caller's inputs are ordered on.
    """

    def __init__(self, n, src, dst, w=None, alpha=0.85, omega=0.8, h_diag=QPR_HDIAG_ZERO,
                 dangling=QPR_DANGLING_F, precision=QPR_FP64, graph_steps=32, stream=None, device=-1,
                 backend=QPR_BACKEND_AUTO, ref_refresh=32, sparse_form=QPR_SPARSE_FORM_AUTO, row_splits=0,
                 adaptive_refresh=1, test_fault=0):
        lib = load_library()
        self._lib = lib
        self.n = int(n)
        src = np.ascontiguousarray(src, dtype=np.int64)
        dst = np.ascontiguousarray(dst, dtype=np.int64)
        self._w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        opt = qpr_options()
        lib.qpr_default_options(ctypes.byref(opt))
        opt.precision, opt.h_diag, opt.dangling = int(precision), int(h_diag), int(dangling)
        opt.graph_steps = int(graph_steps)
        opt.device = int(device)
        opt.backend = int(backend)
        opt.ref_refresh = int(ref_refresh)
        opt.sparse_form = int(sparse_form)
        opt.test_fault = int(test_fault)
        opt.row_splits = int(row_splits)
        opt.adaptive_refresh = int(adaptive_refresh)
        if stream is not None:
            opt.cuda_stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        h = ctypes.c_void_p()
        st = lib.qpr_create(ctypes.byref(h), self.n, int(src.shape[0]), _ptr(src), _ptr(dst),
                            _ptr(self._w), float(alpha), float(omega), ctypes.byref(opt))
        if st != QPR_OK:
            raise QprError(st, lib.qpr_last_error(None).decode())
        self._h = h
        self.alpha, self.omega = float(alpha), float(omega)

    @classmethod
    def from_edges(cls, g, **kw):
        return cls(g.n, g.src, g.dst, g.w, **kw)

    def _raise(self, st):
        if st != QPR_OK:
            raise QprError(st, self._lib.qpr_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.qpr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def backend(self) -> int:
        return int(self._lib.qpr_backend(self._h))

    @property
    def sparse_form(self) -> int:
        """QPR_SPARSE_FORM_COLUMNS, _COLUMNS_PERSISTENT, _COLUMNS_GATHER or
        _TILES (0: not the mixed sparse form)."""
        return int(self._lib.qpr_sparse_form(self._h))

    @property
    def sparse_plan(self) -> dict:
        """Geometry of the column-block product: row splits, complex columns
        per block, CTAs per product launch, shared-memory bytes."""
        out = (ctypes.c_int32 * 4)()
        self._raise(self._lib.qpr_sparse_plan(self._h, out))
        return {"splits": out[0], "block_cols": out[1], "ctas": out[2], "smem": out[3]}

    @property
    def h_spread(self) -> float:
        return float(self._lib.qpr_h_spread(self._h))

    @property
    def max_stable_dt(self) -> float:
        return float(self._lib.qpr_max_stable_dt(self._h))

    def rhs(self, rho, out):
        _check_rho(rho, self.n)
        _check_rho(out, self.n)
        self._raise(self._lib.qpr_rhs(self._h, _ptr(rho), _ptr(out)))
        return out

    def residual(self, rho) -> float:
        _check_rho(rho, self.n)
        r = ctypes.c_double(0.0)
        self._raise(self._lib.qpr_residual(self._h, _ptr(rho), ctypes.byref(r)))
        return float(r.value)

    def evolve(self, rho, dt: float, steps: int):
        """In place: rho <- rho after `steps` RK4 steps."""
        _check_rho(rho, self.n)
        self._raise(self._lib.qpr_evolve(self._h, _ptr(rho), float(dt), int(steps)))
        return rho

    def steady_state(self, rho, dt: float, tol: float, max_steps: int, check: bool = True):
        """In place: rho <- first state with ||f||_F < tol. Returns the stats
        dict (and raises on failure when ``check``)."""
        _check_rho(rho, self.n)
        stats = qpr_stats()
        st = self._lib.qpr_steady_state(self._h, _ptr(rho), float(dt), float(tol), int(max_steps),
                                        ctypes.byref(stats))
        d = stats.as_dict()
        d["status"] = int(st)
        if check and st not in (QPR_OK,):
            self._raise(st)
        return d

    def populations(self, rho, with_rank: bool = False):
        _check_rho(rho, self.n)
        p = np.zeros(self.n)
        rank = np.zeros(self.n, dtype=np.int64) if with_rank else None
        self._raise(self._lib.qpr_populations(self._h, _ptr(rho), _ptr(p), _ptr(rank)))
        return (p, rank) if with_rank else p

    def rkf45(self, rho, tol: float = 1e-8, max_steps: int = 400000, h0: float = 0.0, step_tol: float = 0.0,
              h_max: float = 0.0, t_end: float = 0.0, order: int = 4, check: bool = True):
        """qpr_rkf45 in place on rho: adaptive RKF45 to the steady state
        (t_end <= 0) or to time t_end. Returns the stats dict (with
        "status"); raises on failure when ``check``."""
        _check_rho(rho, self.n)
        opt = qpr_rkf45_options()
        opt.h0, opt.step_tol, opt.h_max, opt.t_end = float(h0), float(step_tol), float(h_max), float(t_end)
        opt.order = int(order)
        stats = qpr_rkf45_stats()
        st = self._lib.qpr_rkf45(self._h, _ptr(rho), ctypes.byref(opt), float(tol), int(max_steps),
                                 ctypes.byref(stats))
        d = stats.as_dict()
        d["status"] = int(st)
        if check and st != QPR_OK:
            self._raise(st)
        return d

    def pagerank(self, tol: float = 1e-14, max_iter: int = 100000, out=None):
        """qpr_pagerank: the classical PageRank vector of the graph (NumPy
        array, or `out` if given: a float64 tensor or array of N entries)."""
        pi = np.zeros(self.n) if out is None else out
        it = ctypes.c_int64(0)
        self._raise(self._lib.qpr_pagerank(self._h, float(tol), int(max_iter), _ptr(pi), ctypes.byref(it)))
        self.last_pagerank_iters = int(it.value)
        return pi

    def hub_classes(self, p, c: float = 10.0):
        """qpr_hub_classes: (classes, counts) of a probability vector p (host
        array or device tensor of N float64); classes is an int32 array."""
        cls = np.zeros(self.n, dtype=np.int32)
        counts = np.zeros(3, dtype=np.int64)
        self._raise(self._lib.qpr_hub_classes(self._h, _ptr(p), float(c), _ptr(cls), _ptr(counts)))
        return cls, counts

    def profile_step(self, rho, dt: float, steps: int):
        """qpr_profile_step: each kernel of `steps` RK4 steps run alone
        between CUDA events; mean durations (ms) of the product, epilogue,
        gain and refresh kernels, and the serialised step."""
        _check_rho(rho, self.n)
        out = qpr_profile()
        self._raise(self._lib.qpr_profile_step(self._h, _ptr(rho), float(dt), int(steps), ctypes.byref(out)))
        return out.as_dict()

    def profile_chain(self, rho, dt: float, reps: int = 20):
        """qpr_profile_chain: the stage-2 SpMM grid and epilogue each
        launched `reps` times back to back with programmatic dependent
        launch; mean time per launch (ms) as {"product_ms", "epilogue_ms"}."""
        _check_rho(rho, self.n)
        out = (ctypes.c_double * 2)()
        self._raise(self._lib.qpr_profile_chain(self._h, _ptr(rho), float(dt), int(reps), out))
        return {"product_ms": out[0], "epilogue_ms": out[1]}


def batch_steady_state(problems, alpha=0.85, dt=0.01, tol=1e-8, max_steps=400000, ref_refresh=32,
                       h_diag=QPR_HDIAG_ZERO, dangling=QPR_DANGLING_F, device=-1, check=True):
    """Batched steady states. ``problems``: list of (EdgeList, omega, rho)
    with rho a complex128 (n, n) torch tensor or NumPy array, overwritten in
    place. Returns (status, list of per-problem stats dicts)."""
    lib = load_library()
    keep = []
    arr = (qpr_problem * len(problems))()
    for i, (g, omega, rho) in enumerate(problems):
        _check_rho(rho, g.n)
        src = np.ascontiguousarray(g.src, dtype=np.int64)
        dst = np.ascontiguousarray(g.dst, dtype=np.int64)
        w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float64)
        keep += [src, dst, w]
        arr[i].n, arr[i].m = int(g.n), int(src.shape[0])
        arr[i].src, arr[i].dst, arr[i].w = _ptr(src), _ptr(dst), _ptr(w)
        arr[i].omega = float(omega)
        arr[i].rho = _ptr(rho)
    opt = qpr_options()
    lib.qpr_default_options(ctypes.byref(opt))
    opt.precision = QPR_MIXED
    opt.ref_refresh, opt.h_diag, opt.dangling, opt.device = int(ref_refresh), int(h_diag), int(dangling), int(device)
    stats = (qpr_stats * len(problems))()
    st = lib.qpr_batch_steady_state(len(problems), arr, float(alpha), float(dt), float(tol), int(max_steps),
                                    ctypes.byref(opt), stats)
    if check and st != QPR_OK:
        raise QprError(st, lib.qpr_last_error(None).decode())
    return st, [stats[i].as_dict() for i in range(len(problems))]


class Gnn:
    """The warm-start network of the C ABI (qpr_gnn_*)."""

    def __init__(self, seed: int = 0, device: int = -1):
        self._lib = load_library()
        h = ctypes.c_void_p()
        st = self._lib.qpr_gnn_create(ctypes.byref(h), int(seed), int(device))
        if st != QPR_OK:
            raise QprError(st, self._lib.qpr_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.qpr_gnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st):
        if st != QPR_OK:
            raise QprError(st, self._lib.qpr_last_error(None).decode())

    @property
    def param_count(self) -> int:
        return int(self._lib.qpr_gnn_param_count())

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count, dtype=np.float32)
        self._raise(self._lib.qpr_gnn_get_params(self._h, _ptr(out)))
        return out

    def set_params(self, params) -> None:
        arr = np.ascontiguousarray(params, dtype=np.float32)
        assert arr.shape == (self.param_count,)
        self._raise(self._lib.qpr_gnn_set_params(self._h, _ptr(arr)))

    def predict(self, g, omega: float, alpha: float = 0.85) -> np.ndarray:
        src = np.ascontiguousarray(g.src, dtype=np.int64)
        dst = np.ascontiguousarray(g.dst, dtype=np.int64)
        w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float64)
        out = np.zeros(g.n)
        self._raise(self._lib.qpr_gnn_predict(self._h, int(g.n), int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(w),
                                              float(alpha), float(omega), _ptr(out)))
        return out

    @staticmethod
    def _samples(samples):
        keep = []
        arr = (qpr_gnn_sample * len(samples))()
        for i, (g, omega, p) in enumerate(samples):
            src = np.ascontiguousarray(g.src, dtype=np.int64)
            dst = np.ascontiguousarray(g.dst, dtype=np.int64)
            w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float64)
            pp = np.ascontiguousarray(p, dtype=np.float64)
            keep += [src, dst, w, pp]
            arr[i].n, arr[i].m = int(g.n), int(src.shape[0])
            arr[i].src, arr[i].dst, arr[i].w, arr[i].p = _ptr(src), _ptr(dst), _ptr(w), _ptr(pp)
            arr[i].omega = float(omega)
        return arr, keep

    def loss_grad(self, g, omega, p, alpha=0.85):
        arr, keep = self._samples([(g, omega, p)])
        loss = ctypes.c_double(0.0)
        grad = np.zeros(self.param_count, dtype=np.float32)
        self._raise(self._lib.qpr_gnn_loss_grad(self._h, arr, float(alpha), ctypes.byref(loss), _ptr(grad)))
        return float(loss.value), grad

    def train(self, samples, epochs=20, batch=8, lr=1e-3, seed=0, alpha=0.85):
        arr, keep = self._samples(samples)
        losses = np.zeros(int(epochs))
        self._raise(self._lib.qpr_gnn_train(self._h, len(samples), arr, float(alpha), int(epochs), int(batch),
                                            float(lr), int(seed), _ptr(losses)))
        return losses


def tuned_options(r) -> dict:
    """Solver keyword options of an autotune result."""
    return {"backend": r["backend"], "ref_refresh": r["ref_refresh"], "sparse_form": r["sparse_form"],
            "row_splits": r["row_splits"]}


def autotune(g, omega, alpha=0.85, dt=0.01, precision=QPR_MIXED, cache_path=None, device=-1):
    """qpr_autotune for an EdgeList: returns dict(backend, ref_refresh,
    ms_per_step, from_cache, sparse_form, row_splits); Solver(...,
    **tuned_options(result)) runs the chosen configuration."""
    lib = load_library()
    src = np.ascontiguousarray(g.src, dtype=np.int64)
    dst = np.ascontiguousarray(g.dst, dtype=np.int64)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float64)
    opt = qpr_options()
    lib.qpr_default_options(ctypes.byref(opt))
    opt.precision, opt.device = int(precision), int(device)
    res = qpr_tune_result()
    st = lib.qpr_autotune(int(g.n), int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(w), float(alpha), float(omega),
                          float(dt), ctypes.byref(opt), None if cache_path is None else str(cache_path).encode(),
                          ctypes.byref(res))
    if st != QPR_OK:
        raise QprError(st, lib.qpr_last_error(None).decode())
    return {"backend": res.backend, "ref_refresh": res.ref_refresh, "ms_per_step": res.ms_per_step,
            "from_cache": res.from_cache, "sparse_form": res.sparse_form, "row_splits": res.row_splits}
