"""ctypes wrapper of the plain FP64 C oracle (``qpr_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qpr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libqpr_oracle.so")

OR_OK, OR_E_ARG, OR_E_GRAPH, OR_E_OOM, OR_E_NOT_CONVERGED, OR_E_NONFINITE = 0, 1, 2, 4, 6, 8


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what} failed with status {status}")
        self.status = status


def oracle_lib_path() -> str:
    return _LIB


def build_oracle_lib(force: bool = False) -> str:
    """Compile ``qpr_oracle.c`` with gcc (OpenMP, no fast-math, no FMA
    contraction so that x86 and Arm hosts give identical results)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build_oracle_lib()
        lib = ctypes.CDLL(_LIB)
        i64, f64, vp, ip = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
        lib.oracle_create.restype = vp
        lib.oracle_create.argtypes = [i64, i64, vp, vp, vp, f64, f64, ip, ip, ctypes.POINTER(ip)]
        lib.oracle_free.argtypes = [vp]
        lib.oracle_n.restype = i64
        lib.oracle_n.argtypes = [vp]
        lib.oracle_h_nnz.restype = i64
        lib.oracle_h_nnz.argtypes = [vp]
        lib.oracle_dropped_self_loops.restype = i64
        lib.oracle_dropped_self_loops.argtypes = [vp]
        lib.oracle_get_operators.argtypes = [vp, vp, vp, vp, vp]
        lib.oracle_rhs.argtypes = [vp, vp, vp]
        lib.oracle_residual.restype = f64
        lib.oracle_residual.argtypes = [vp, vp]
        lib.oracle_prepare.restype = f64
        lib.oracle_prepare.argtypes = [i64, vp]
        lib.oracle_evolve.restype = ip
        lib.oracle_evolve.argtypes = [vp, vp, f64, i64]
        lib.oracle_steady_state.restype = ip
        lib.oracle_steady_state.argtypes = [vp, vp, f64, f64, i64, ctypes.POINTER(i64),
                                            ctypes.POINTER(f64), vp]
        lib.oracle_rkf45.restype = ip
        lib.oracle_rkf45.argtypes = [vp, vp, f64, f64, f64, f64, f64, i64, ip, ctypes.POINTER(i64),
                                     ctypes.POINTER(i64), ctypes.POINTER(f64), ctypes.POINTER(f64),
                                     ctypes.POINTER(f64), vp, i64]
        lib.oracle_rkf45_step.restype = f64
        lib.oracle_rkf45_step.argtypes = [vp, vp, f64, vp, vp]
        lib.oracle_set_threads.argtypes = [ip]
        lib.oracle_max_threads.restype = ip
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


class Oracle:
    """FP64 CPU oracle of one problem (graph, alpha, omega, modes)."""

    def __init__(self, n, src, dst, w=None, alpha=0.85, omega=0.8, h_diag=0, dangling=0):
        lib = _load()
        self._lib = lib
        self.n = int(n)
        src = np.ascontiguousarray(src, dtype=np.int64)
        dst = np.ascontiguousarray(dst, dtype=np.int64)
        wp = None
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float64)
            wp = _ptr(w)
        st = ctypes.c_int(0)
        h = lib.oracle_create(self.n, int(src.shape[0]), _ptr(src), _ptr(dst), wp,
                              float(alpha), float(omega), int(h_diag), int(dangling),
                              ctypes.byref(st))
        if not h:
            raise OracleError(st.value, "create")
        self._h = h
        self.alpha, self.omega = float(alpha), float(omega)

    @classmethod
    def from_edges(cls, g, **kw):
        return cls(g.n, g.src, g.dst, g.w, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def operators(self):
        """(A, H, G, c) as float64 arrays."""
        n = self.n
        A = np.zeros((n, n)); H = np.zeros((n, n)); G = np.zeros((n, n)); c = np.zeros(n)
        self._lib.oracle_get_operators(self._h, _ptr(A), _ptr(H), _ptr(G), _ptr(c))
        return A, H, G, c

    @property
    def h_nnz(self) -> int:
        return int(self._lib.oracle_h_nnz(self._h))

    def rhs(self, rho: np.ndarray) -> np.ndarray:
        rho = np.ascontiguousarray(rho, dtype=np.complex128)
        out = np.empty_like(rho)
        self._lib.oracle_rhs(self._h, _ptr(rho), _ptr(out))
        return out

    def residual(self, rho: np.ndarray) -> float:
        rho = np.ascontiguousarray(rho, dtype=np.complex128)
        return float(self._lib.oracle_residual(self._h, _ptr(rho)))

    def evolve(self, rho0: np.ndarray, dt: float, steps: int) -> np.ndarray:
        y = np.array(rho0, dtype=np.complex128, order="C", copy=True)
        st = self._lib.oracle_evolve(self._h, _ptr(y), float(dt), int(steps))
        if st != OR_OK:
            raise OracleError(st, "evolve")
        return y

    def steady_state(self, rho0: np.ndarray, dt: float, tol: float, max_steps: int,
                     history: bool = False):
        """Returns (rho, steps, residual, status[, residual history])."""
        y = np.array(rho0, dtype=np.complex128, order="C", copy=True)
        steps = ctypes.c_int64(0)
        r = ctypes.c_double(0.0)
        hist = np.zeros(int(max_steps) + 1) if history else None
        st = self._lib.oracle_steady_state(self._h, _ptr(y), float(dt), float(tol), int(max_steps),
                                           ctypes.byref(steps), ctypes.byref(r),
                                           _ptr(hist) if history else None)
        if st not in (OR_OK, OR_E_NOT_CONVERGED):
            raise OracleError(st, "steady_state")
        out = (y, int(steps.value), float(r.value), int(st))
        if history:
            out = out + (hist[: int(steps.value) + 1],)
        return out

    def rkf45(self, rho0: np.ndarray, h0: float, step_tol: float, h_max: float, resid_tol: float = 0.0,
              t_end: float = float("inf"), max_steps: int = 10**7, history: bool = False, hist_cap: int = 200000,
              order: int = 4):
        """Adaptive RKF45 (Supplementary Note 2, Eq. S10 - S13; readings in
        qpr_oracle.c; order 4 propagates y_{k+1} of Eq. S11, order 5 the
        alternative z_{k+1} of Eq. S12). Returns a dict: rho, accepted, rejected, t, h (the next
        attempt's step), residual, status, and with ``history`` an array of
        (t, h, discrepancy, s, accepted) per attempt."""
        y = np.array(rho0, dtype=np.complex128, order="C", copy=True)
        acc, rej = ctypes.c_int64(0), ctypes.c_int64(0)
        t, h, r = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        hist = np.zeros((hist_cap, 5)) if history else None
        st = self._lib.oracle_rkf45(self._h, _ptr(y), float(h0), float(step_tol), float(h_max), float(resid_tol),
                                    float(t_end), int(max_steps), int(order), ctypes.byref(acc), ctypes.byref(rej),
                                    ctypes.byref(t), ctypes.byref(h), ctypes.byref(r),
                                    _ptr(hist) if history else None, int(hist_cap) if history else 0)
        if st not in (OR_OK, OR_E_NOT_CONVERGED):
            raise OracleError(st, "rkf45")
        out = {"rho": y, "accepted": int(acc.value), "rejected": int(rej.value), "t": float(t.value),
               "h": float(h.value), "residual": float(r.value), "status": int(st)}
        if history:
            out["history"] = hist[: min(hist_cap, out["accepted"] + out["rejected"])]
        return out

    def rkf45_step(self, rho: np.ndarray, h: float):
        """One RKF45 attempt without step-size control from rho (used as
        given): (y_{k+1} of Eq. S11, z_{k+1} of Eq. S12, |z - y|)."""
        rho = np.ascontiguousarray(rho, dtype=np.complex128)
        y4 = np.empty_like(rho)
        z5 = np.empty_like(rho)
        err = self._lib.oracle_rkf45_step(self._h, _ptr(rho), float(h), _ptr(y4), _ptr(z5))
        return y4, z5, float(err)


def prepare(rho: np.ndarray) -> np.ndarray:
    """(rho + rho^dag)/2 divided by its real trace, as the oracle does."""
    y = np.array(rho, dtype=np.complex128, order="C", copy=True)
    _load().oracle_prepare(y.shape[0], _ptr(y))
    return y


def populations(rho: np.ndarray) -> np.ndarray:
    """p_i = Re rho_ii (the probability at node i)."""
    return np.real(np.diag(rho)).copy()


def ranking(p: np.ndarray) -> np.ndarray:
    """Node indices by descending probability; ties go to the lower index."""
    return np.argsort(-np.asarray(p), kind="stable")


def hub_classes(p: np.ndarray, c: float = 10.0) -> np.ndarray:
    """0 = rest, 1 = secondary hub (1/N < p <= c/N), 2 = main hub (p > c/N).

    Thresholds follow the main text's definition of hubs (Sec. on the airline
    ranking); the text does not say which side the equalities fall on.
    """
    p = np.asarray(p)
    n = p.shape[0]
    out = np.zeros(n, dtype=np.int64)
    out[(p > 1.0 / n) & (p <= c / n)] = 1
    out[p > c / n] = 2
    return out
