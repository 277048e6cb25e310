"""Thin Python binding of the C ABI in include/ptp.h (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library libptp.so.  Tensors are torch CUDA tensors (device memory) or numpy
arrays (host memory); streams are torch.cuda.Stream objects or None for the
current stream.  The library must have been built (build.build()); loading
fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PTP_OK = 0
PTP_ERR_ARG = 1
PTP_ERR_INDEX = 2
PTP_ERR_DEGENERATE_FACE = 3
PTP_ERR_CUDA = 4
PTP_ERR_NOT_CONVERGED = 5
PTP_ERR_TIMEOUT = 6
PTP_ERR_NOMEM = 7
PTP_ERR_TOO_LARGE = 8

PTP_HOST = 0
PTP_DEVICE = 1

_lock = threading.Lock()
_lib = None


class PTPError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)}")


class Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("eps_abs", ctypes.c_double), ("max_iter", ctypes.c_int64),
                ("block", ctypes.c_int32), ("grid", ctypes.c_int32), ("band_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_int64),
                ("ev_begin", ctypes.c_void_p), ("ev_end", ctypes.c_void_p), ("schedule", ctypes.c_void_p),
                ("mlp_half", ctypes.c_void_p), ("mlp_margin", ctypes.c_float), ("reserved2", ctypes.c_int32),
                ("conv_trace", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("band_updates", ctypes.c_int64), ("active_updates", ctypes.c_int64),
                ("changed", ctypes.c_int64), ("fp64_solves", ctypes.c_int64), ("rho", ctypes.c_int32),
                ("status", ctypes.c_int32), ("checks", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("grid", ctypes.c_int32), ("ms", ctypes.c_float),
                ("ms_default", ctypes.c_float), ("tried", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


TRACE_DTYPE = np.dtype([("i", np.int32), ("j", np.int32), ("active", np.int32), ("changed", np.int32),
                        ("maxrel", np.float32), ("advanced", np.int32), ("errsum", np.float64)])


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libptp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_1810_08218_gb300.build.build())")
        lib = ctypes.CDLL(p)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int32
        st = ctypes.c_int
        sig = {
            "ptp_status_str": (ctypes.c_char_p, [st]),
            "ptp_params_default": (st, [P]),
            "ptp_kernel_launches": (i64, []),
            "ptp_release_memory": (st, []),
            "ptp_mesh_create": (st, [P, i64, P, i64, ctypes.c_int, P, P]),
            "ptp_mesh_info": (st, [P, P, P, P]),
            "ptp_mesh_destroy": (st, [P]),
            "ptp_toplesets": (st, [P, P, i32, ctypes.c_int, P, P]),
            "ptp_toplesets_info": (st, [P, P, P, P, P, P]),
            "ptp_toplesets_destroy": (st, [P]),
            "ptp_distance": (st, [P, P, P, P, P]),
            "ptp_last_stats": (st, [P, P, P]),
            "ptp_distance_noalloc": (st, [P, P, P, P, P]),
            "ptp_distance_from_sources": (st, [P, P, i32, ctypes.c_int, P, P, P, P]),
            "ptp_batch_create": (st, [P, i32, P, P]),
            "ptp_distance_batch": (st, [P, P, P, P, P]),
            "ptp_batch_destroy": (st, [P]),
            "ptp_autotune": (st, [P, P, P, i32, P, P]),
            "ptp_selftest_wait_limit": (st, [i64, P]),
            "ptp_voronoi": (st, [P, P, i32, ctypes.c_int, P, P, P, P, P]),
            "ptp_window_features": (st, [P, P, P]),
            "ptp_mlp_infer": (st, [P, P, i32, P, ctypes.c_float, i32, P, P]),
            "ptp_mlp_grad": (st, [P, P, P, i32, P, P, P]),
            "ptp_mlp_adam": (st, [P, P, P, P, P, ctypes.c_float, i32, P]),
            "ptp_mlp_to_half": (st, [P, P, P]),
            "ptp_fps": (st, [P, i32, i32, P, P, P, ctypes.c_int, P, P]),
            "ptp_geodesic": (st, [P, i64, P, i64, P, i32, ctypes.c_int, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_str(code: int) -> str:
    try:
        return load().ptp_status_str(int(code)).decode()
    except Exception:
        return f"status {code}"


def _check(code: int, where: str, ok=(PTP_OK,)):
    if code not in ok:
        raise PTPError(code, where)
    return code


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def _stream_ptr(stream) -> int | None:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def _array_arg(x, dtype):
    """(pointer, ptr_kind, keepalive) for a torch CUDA tensor or a host array."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        kind = PTP_DEVICE if x.is_cuda else PTP_HOST
        return ctypes.c_void_p(x.data_ptr()), kind, x
    a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), PTP_HOST, a


class _DevView:
    """Exposes a device pointer through __cuda_array_interface__ so torch can
    wrap it without a copy (the owning handle must stay alive)."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}
        self._owner = owner


# --------------------------------------------------------------------------
# handles
# --------------------------------------------------------------------------

class Mesh:
    def __init__(self, handle: ctypes.c_void_p, n: int, nf: int, diameter: float):
        self.handle = handle
        self.n = n
        self.nf = nf
        self.diameter = diameter

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                ptp_mesh_destroy(self)
            except Exception:
                pass


class Toplesets:
    def __init__(self, handle: ctypes.c_void_p, mesh: Mesh):
        self.handle = handle
        self.mesh = mesh  # keeps the mesh alive

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                ptp_toplesets_destroy(self)
            except Exception:
                pass


class Batch:
    def __init__(self, handle: ctypes.c_void_p, sizes: list[int]):
        self.handle = handle
        self.sizes = sizes  # vertices per map

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                ptp_batch_destroy(self)
            except Exception:
                pass


# --------------------------------------------------------------------------
# the C ABI, same names
# --------------------------------------------------------------------------

def ptp_params_default(**overrides) -> Params:
    p = Params()
    _check(load().ptp_params_default(ctypes.byref(p)), "ptp_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def ptp_kernel_launches() -> int:
    return int(load().ptp_kernel_launches())


def ptp_release_memory() -> None:
    """Trim the library's device memory pools to what is still in use."""
    _check(load().ptp_release_memory(), "ptp_release_memory")


def ptp_mesh_create(xyz, faces, stream=None) -> Mesh:
    lib = load()
    px, kx, kx_keep = _array_arg(xyz, np.float32)
    pf, kf, kf_keep = _array_arg(faces, np.int32)
    if kx != kf:
        raise ValueError("xyz and faces must both be host arrays or both device tensors")
    n = int(np.prod(kx_keep.shape)) // 3
    nf = int(np.prod(kf_keep.shape)) // 3
    h = ctypes.c_void_p()
    _check(lib.ptp_mesh_create(px, n, pf, nf, kx, _stream_ptr(stream), ctypes.byref(h)), "ptp_mesh_create")
    d = ctypes.c_double()
    lib.ptp_mesh_info(h, None, None, ctypes.byref(d))
    return Mesh(h, n, nf, d.value)


def ptp_mesh_info(mesh: Mesh) -> tuple[int, int, float]:
    n = ctypes.c_int64()
    nf = ctypes.c_int64()
    d = ctypes.c_double()
    _check(load().ptp_mesh_info(mesh.handle, ctypes.byref(n), ctypes.byref(nf), ctypes.byref(d)), "ptp_mesh_info")
    return n.value, nf.value, d.value


def ptp_mesh_destroy(mesh: Mesh) -> None:
    if mesh.handle:
        h, mesh.handle = mesh.handle, None
        _check(load().ptp_mesh_destroy(h), "ptp_mesh_destroy")


def ptp_toplesets(mesh: Mesh, sources, stream=None) -> Toplesets:
    lib = load()
    ps, ks, keep = _array_arg(sources, np.int32)
    m = int(np.prod(keep.shape))
    h = ctypes.c_void_p()
    _check(lib.ptp_toplesets(mesh.handle, ps, m, ks, _stream_ptr(stream), ctypes.byref(h)), "ptp_toplesets")
    return Toplesets(h, mesh)


def ptp_toplesets_info(tops: Toplesets, stream=None) -> dict:
    """rho, n_reached and (as torch int32 CUDA tensors viewing the handle's
    memory) the topleset offsets [rho+1] and the permutation [n]."""
    import torch

    rho = ctypes.c_int32()
    nr = ctypes.c_int32()
    off = ctypes.c_void_p()
    perm = ctypes.c_void_p()
    _check(load().ptp_toplesets_info(tops.handle, _stream_ptr(stream), ctypes.byref(rho), ctypes.byref(nr),
                                     ctypes.byref(off), ctypes.byref(perm)), "ptp_toplesets_info")
    offt = torch.as_tensor(_DevView(off.value, rho.value + 1, "<i4", tops), device="cuda")
    permt = torch.as_tensor(_DevView(perm.value, tops.mesh.n, "<i4", tops), device="cuda")
    return {"rho": rho.value, "n_reached": nr.value, "off": offt, "perm": permt}


def ptp_toplesets_destroy(tops: Toplesets) -> None:
    if tops.handle:
        h, tops.handle = tops.handle, None
        _check(load().ptp_toplesets_destroy(h), "ptp_toplesets_destroy")


def ptp_distance(tops: Toplesets, params: Params, d_out, stream=None, stats: bool = True,
                 ok=(PTP_OK,)) -> dict | None:
    """Fill d_out (torch float32 CUDA tensor [n], original vertex order).
    With stats=True the call blocks and returns the run statistics."""
    st = Stats() if stats else None
    code = load().ptp_distance(tops.handle, ctypes.byref(params), ctypes.c_void_p(d_out.data_ptr()),
                               _stream_ptr(stream), ctypes.byref(st) if st is not None else None)
    _check(code, "ptp_distance", ok)
    return st.as_dict() if st is not None else None


def ptp_distance_noalloc(tops: Toplesets, params: Params, d_out, stream=None, stats: bool = True,
                         ok=(PTP_OK,)) -> dict | None:
    """ptp_distance with its scratch in the library's static device array
    (no allocation; at most PTP_NOALLOC_MAX_VERTS vertices)."""
    st = Stats() if stats else None
    code = load().ptp_distance_noalloc(tops.handle, ctypes.byref(params), ctypes.c_void_p(d_out.data_ptr()),
                                       _stream_ptr(stream), ctypes.byref(st) if st is not None else None)
    _check(code, "ptp_distance_noalloc", ok)
    return st.as_dict() if st is not None else None


PTP_NOALLOC_MAX_VERTS = 1048576


def ptp_distance_from_sources(mesh: Mesh, sources, params: Params, d_out, stream=None, stats: bool = True,
                              ok=(PTP_OK,)) -> dict | None:
    """The map from a mesh and a source set in one fused launch (toplesets
    built while the iteration runs); d_out float32 CUDA tensor [n]."""
    ps, ks, keep = _array_arg(sources, np.int32)
    st = Stats() if stats else None
    code = load().ptp_distance_from_sources(mesh.handle, ps, int(np.prod(keep.shape)), ks, ctypes.byref(params),
                                            ctypes.c_void_p(d_out.data_ptr()), _stream_ptr(stream),
                                            ctypes.byref(st) if st is not None else None)
    _check(code, "ptp_distance_from_sources", ok)
    return st.as_dict() if st is not None else None


PTP_BATCH_MAX = 32


def ptp_batch_create(tops: list[Toplesets], stream=None) -> Batch:
    """Concatenate up to PTP_BATCH_MAX toplesets handles into one batch."""
    arr = (ctypes.c_void_p * len(tops))(*[t.handle.value if isinstance(t.handle, ctypes.c_void_p) else t.handle
                                          for t in tops])
    h = ctypes.c_void_p()
    _check(load().ptp_batch_create(arr, len(tops), _stream_ptr(stream), ctypes.byref(h)), "ptp_batch_create")
    return Batch(h, [t.mesh.n for t in tops])


def ptp_batch_destroy(batch: Batch) -> None:
    h, batch.handle = batch.handle, None
    if h:
        _check(load().ptp_batch_destroy(h), "ptp_batch_destroy")


def ptp_distance_batch(batch: Batch, params: Params, d_outs, stream=None, stats: bool = True,
                       ok=(PTP_OK,)) -> list[dict] | None:
    """All maps of the batch in one launch; d_outs[b] is a float32 CUDA
    tensor of map b's vertex count.  Returns per-map statistics."""
    if len(d_outs) != len(batch.sizes):
        raise ValueError("one output per map")
    ptrs = (ctypes.c_void_p * len(d_outs))(*[d.data_ptr() for d in d_outs])
    st = (Stats * len(d_outs))() if stats else None
    code = load().ptp_distance_batch(batch.handle, ctypes.byref(params), ptrs, _stream_ptr(stream),
                                     st if st is not None else None)
    _check(code, "ptp_distance_batch", ok)
    return [x.as_dict() for x in st] if st is not None else None


def ptp_autotune(target, params: Params, reps: int = 3, stream=None) -> dict:
    """Time the window kernel's launch shapes on `target` (a Toplesets or a
    Batch), write the fastest into params.block / params.grid and return
    the timings."""
    r = TuneResult()
    tops = target.handle if isinstance(target, Toplesets) else None
    batch = target.handle if isinstance(target, Batch) else None
    _check(load().ptp_autotune(tops, batch, ctypes.byref(params), reps, _stream_ptr(stream), ctypes.byref(r)),
           "ptp_autotune")
    return r.as_dict()


def ptp_selftest_wait_limit(cycles: int, stream=None) -> int:
    """Status of a launch whose only wait can end by its limit alone
    (PTP_ERR_TIMEOUT when the limit works)."""
    return int(load().ptp_selftest_wait_limit(int(cycles), _stream_ptr(stream)))


def ptp_voronoi(mesh: Mesh, seeds, params: Params, d_out=None, label_out=None, stream=None, stats: bool = True,
                ok=(PTP_OK,)) -> dict | None:
    """Multi-source map from `seeds` with the index of the nearest seed per
    vertex (torch CUDA tensors: d_out float32 [n], label_out int32 [n])."""
    ps, ks, keep = _array_arg(seeds, np.int32)
    st = Stats() if stats else None
    code = load().ptp_voronoi(mesh.handle, ps, int(np.prod(keep.shape)), ks, ctypes.byref(params),
                              ctypes.c_void_p(d_out.data_ptr()) if d_out is not None else None,
                              ctypes.c_void_p(label_out.data_ptr()) if label_out is not None else None,
                              _stream_ptr(stream), ctypes.byref(st) if st is not None else None)
    _check(code, "ptp_voronoi", ok)
    return st.as_dict() if st is not None else None


def ptp_fps(mesh: Mesh, first: int, n_samples: int, params: Params, samples_out, d_out=None, use_graph: bool = True,
            stream=None, stats: bool = True, ok=(PTP_OK,)) -> dict | None:
    """Farthest-point sampling on the device (samples_out: int32 CUDA tensor
    [n_samples]; d_out: optional float32 CUDA tensor [n])."""
    st = Stats() if stats else None
    code = load().ptp_fps(mesh.handle, int(first), int(n_samples), ctypes.byref(params),
                          ctypes.c_void_p(samples_out.data_ptr()),
                          ctypes.c_void_p(d_out.data_ptr()) if d_out is not None else None, 1 if use_graph else 0,
                          _stream_ptr(stream), ctypes.byref(st) if st is not None else None)
    _check(code, "ptp_fps", ok)
    return st.as_dict() if st is not None else None


def ptp_last_stats(tops: Toplesets, stream=None) -> dict:
    st = Stats()
    load().ptp_last_stats(tops.handle, _stream_ptr(stream), ctypes.byref(st))
    return st.as_dict()


def ptp_geodesic(xyz, faces, sources, params: Params, d_out, stream=None, ok=(PTP_OK,)) -> dict:
    """Whole pipeline in one call.  All arrays must be of one kind: host
    (numpy / CPU tensors, d_out a writable float32 host array) or device."""
    lib = load()
    px, kx, kx_keep = _array_arg(xyz, np.float32)
    pf, kf, kf_keep = _array_arg(faces, np.int32)
    ps, ks, ks_keep = _array_arg(sources, np.int32)
    try:
        import torch
        is_t = isinstance(d_out, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_t = False
    if is_t:
        pd, kd = ctypes.c_void_p(d_out.data_ptr()), (PTP_DEVICE if d_out.is_cuda else PTP_HOST)
    else:
        if not (isinstance(d_out, np.ndarray) and d_out.dtype == np.float32 and d_out.flags.c_contiguous):
            raise ValueError("host d_out must be a contiguous float32 numpy array")
        pd, kd = d_out.ctypes.data_as(ctypes.c_void_p), PTP_HOST
    if len({kx, kf, ks, kd}) != 1:
        raise ValueError("xyz, faces, sources and d_out must all be host or all device")
    n = int(np.prod(kx_keep.shape)) // 3
    nf = int(np.prod(kf_keep.shape)) // 3
    m = int(np.prod(ks_keep.shape))
    st = Stats()
    code = lib.ptp_geodesic(px, n, pf, nf, ps, m, kx, ctypes.byref(params), pd, _stream_ptr(stream),
                            ctypes.byref(st))
    _check(code, "ptp_geodesic", ok)
    return st.as_dict()


# --------------------------------------------------------------------------
# learned schedule (MLP kernels)
# --------------------------------------------------------------------------

PTP_MLP_NPARAM = 1313
PTP_WINDOW_FEATURES = 6


def _dp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def ptp_window_features(tops: Toplesets, feat_out, stream=None) -> None:
    """feat_out: float32 CUDA tensor with room for 6 * n floats."""
    _check(load().ptp_window_features(tops.handle, _dp(feat_out), _stream_ptr(stream)), "ptp_window_features")


def ptp_mlp_infer(w_half, feat, count: int, sched_out, margin: float = 0.0, cap: int = 1 << 20, count_dev=None,
                  stream=None) -> None:
    _check(load().ptp_mlp_infer(_dp(w_half), _dp(feat), int(count), _dp(count_dev), float(margin), int(cap),
                                _dp(sched_out), _stream_ptr(stream)), "ptp_mlp_infer")


def ptp_mlp_grad(w_half, X, Y, count: int, grad, loss=None, stream=None) -> None:
    _check(load().ptp_mlp_grad(_dp(w_half), _dp(X), _dp(Y), int(count), _dp(grad), _dp(loss), _stream_ptr(stream)),
           "ptp_mlp_grad")


def ptp_mlp_adam(w_master, w_half, m, v, grad, lr: float, step: int, stream=None) -> None:
    _check(load().ptp_mlp_adam(_dp(w_master), _dp(w_half), _dp(m), _dp(v), _dp(grad), float(lr), int(step),
                               _stream_ptr(stream)), "ptp_mlp_adam")


def ptp_mlp_to_half(w, w_half, stream=None) -> None:
    _check(load().ptp_mlp_to_half(_dp(w), _dp(w_half), _stream_ptr(stream)), "ptp_mlp_to_half")

