"""FP64 CPU oracle for Parallel Toplesets Propagation (PTP).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  Nothing in the library
imports this package, and this package imports nothing from the library.

The arithmetic lives in ``ptp_oracle.c`` (plain single-threaded C, FP64),
compiled with gcc into ``oracle/_build/libptp_oracle.so`` on first use or by
``build()``.  Each C function cites the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libptp_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
NOT_CONVERGED = 1
ERR_ARG = -1
ERR_INDEX = -2
ERR_DEGENERATE_FACE = -3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, no FMA contraction, no
    target flags, so x86 and Arm builds round identically)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            i32 = ctypes.c_int32
            dbl = ctypes.c_double
            lib.or_update.restype = dbl
            lib.or_update.argtypes = [P, P, P, dbl, dbl]
            lib.or_incident.restype = ctypes.c_int
            lib.or_incident.argtypes = [i64, i64, P, P, P, P]
            lib.or_toplesets.restype = i64
            lib.or_toplesets.argtypes = [i64, P, P, P, i32, P, P]
            lib.or_ptp.restype = ctypes.c_int
            lib.or_ptp.argtypes = [i64, P, i64, P, i32, P, dbl, dbl, i64, ctypes.c_int, P, P, P, P, P, i64, P, i64]
            lib.or_relax.restype = i64
            lib.or_relax.argtypes = [i64, P, i64, P, i32, P, ctypes.c_int, ctypes.c_uint64, i64, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def update(x0, x1, x2, d1: float, d2: float) -> float:
    """The per-triangle update step (Sec. 3.2) for vertex x0."""
    lib = _load()
    a0 = np.ascontiguousarray(x0, dtype=np.float64)
    a1 = np.ascontiguousarray(x1, dtype=np.float64)
    a2 = np.ascontiguousarray(x2, dtype=np.float64)
    return float(lib.or_update(_ptr(a0), _ptr(a1), _ptr(a2), float(d1), float(d2)))


def incident(n: int, F: np.ndarray):
    """Vertex -> incident triangles: (row[n+1], a[3nf], b[3nf])."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.int32)
    row = np.zeros(n + 1, dtype=np.int64)
    oa = np.zeros(3 * F.shape[0], dtype=np.int32)
    ob = np.zeros(3 * F.shape[0], dtype=np.int32)
    rc = lib.or_incident(n, F.shape[0], _ptr(F), _ptr(row), _ptr(oa), _ptr(ob))
    if rc != OK:
        raise ValueError(f"or_incident failed: {rc}")
    return row, oa, ob


def toplesets(n: int, F: np.ndarray, sources) -> tuple[np.ndarray, int]:
    """BFS levels (topleset index per vertex, -1 if unreachable) and rho."""
    lib = _load()
    row, oa, ob = incident(n, F)
    src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
    level = np.zeros(n, dtype=np.int32)
    rho = lib.or_toplesets(n, _ptr(row), _ptr(oa), _ptr(ob), src.shape[0], _ptr(src), _ptr(level))
    if rho < 0:
        raise ValueError(f"or_toplesets failed: {rho}")
    return level, int(rho)


class PTPResult:
    """Oracle output: distances, K, rho, vertex updates, status, traces."""

    def __init__(self, d, stats, ti, tj, tm, hist):
        self.d = d
        self.K = int(stats[0])
        self.rho = int(stats[1])
        self.updates = int(stats[2])
        self.status = int(stats[3])
        self.trace_i = ti
        self.trace_j = tj
        self.trace_maxrel = tm
        self.hist = hist


def ptp(V: np.ndarray, F: np.ndarray, sources, eps: float = 1e-3, eps_abs: float = 0.0,
        max_iter: int = 0, trace: bool = False, history: int = 0, band_mode: int = 0) -> PTPResult:
    """Run the oracle PTP (Sec. 4.2) in FP64.  `history` > 0 keeps d_k for
    k = 0 .. history-1 (tiny meshes only).  band_mode 1: the fixed band of
    the complexity analysis (Sec. 6.1) instead of Eq. lower_band."""
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
    n = V.shape[0]
    d = np.zeros(n, dtype=np.float64)
    stats = np.zeros(4, dtype=np.int64)
    cap = 0
    ti = tj = tm = None
    if trace:
        cap = max_iter if max_iter > 0 else 8 * n + 64
        ti = np.full(cap, -1, dtype=np.int32)
        tj = np.full(cap, -1, dtype=np.int32)
        tm = np.zeros(cap, dtype=np.float64)
    hist = np.zeros((history, n), dtype=np.float64) if history > 0 else None
    rc = lib.or_ptp(n, _ptr(V), F.shape[0], _ptr(F), src.shape[0], _ptr(src), float(eps), float(eps_abs),
                    int(max_iter), int(band_mode), _ptr(d), _ptr(stats),
                    _ptr(ti) if ti is not None else None, _ptr(tj) if tj is not None else None,
                    _ptr(tm) if tm is not None else None, cap,
                    _ptr(hist) if hist is not None else None, history)
    if rc < 0:
        raise ValueError(f"or_ptp failed: {rc}")
    if trace:
        K = int(stats[0])
        ti, tj, tm = ti[:K], tj[:K], tm[:K]
    return PTPResult(d, stats, ti, tj, tm, hist)


def relax(V: np.ndarray, F: np.ndarray, sources, mode: int = 0, seed: int = 0,
          max_sweeps: int = 100000) -> tuple[np.ndarray, int]:
    """Full relaxation to the update operator's fixpoint.  mode 0 Jacobi,
    1 Gauss-Seidel in index order, 2 Gauss-Seidel in seeded random order."""
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
    d = np.zeros(V.shape[0], dtype=np.float64)
    sweeps = lib.or_relax(V.shape[0], _ptr(V), F.shape[0], _ptr(F), src.shape[0], _ptr(src),
                          int(mode), int(seed), int(max_sweeps), _ptr(d))
    if sweeps < 0:
        raise ValueError(f"or_relax failed: {sweeps}")
    return d, int(sweeps)
