"""The C ABI library loads and exports every function include/ptp.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

from paper_1810_08218_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(ptp_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("ptp_mesh_create", "ptp_toplesets", "ptp_distance", "ptp_geodesic", "ptp_status_str"):
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    lib.ptp_status_str.restype = ctypes.c_char_p
    assert lib.ptp_status_str(0) == b"PTP_OK"
    assert lib.ptp_status_str(6) == b"PTP_ERR_TIMEOUT"
    from paper_1810_08218_gb300 import capi

    p = capi.Params()
    assert lib.ptp_params_default(ctypes.byref(p)) == 0
    assert p.eps == 1e-3 and p.eps_abs == 0.0 and p.max_iter == 0
    # argument errors are reported before any CUDA call
    out = ctypes.c_void_p()
    assert lib.ptp_mesh_create(None, 10, None, 1, 0, None, ctypes.byref(out)) == capi.PTP_ERR_ARG
    assert lib.ptp_params_default(None) == capi.PTP_ERR_ARG
    # no pool has been created in a process without CUDA work: nothing to trim
    assert lib.ptp_release_memory() == 0


def test_batch_argument_errors_before_cuda(lib):
    from paper_1810_08218_gb300 import capi

    out = ctypes.c_void_p()
    lib.ptp_batch_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.ptp_batch_create(None, 1, None, ctypes.byref(out)) == capi.PTP_ERR_ARG
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.ptp_batch_create(arr, 1, None, ctypes.byref(out)) == capi.PTP_ERR_ARG
    assert lib.ptp_batch_create(arr, 0, None, ctypes.byref(out)) == capi.PTP_ERR_ARG
    assert lib.ptp_batch_create(arr, 33, None, ctypes.byref(out)) == capi.PTP_ERR_ARG
    assert lib.ptp_batch_create(arr, 1, None, None) == capi.PTP_ERR_ARG
    lib.ptp_distance_batch.argtypes = [ctypes.c_void_p] * 5
    p = capi.Params()
    assert lib.ptp_distance_batch(None, ctypes.byref(p), None, None, None) == capi.PTP_ERR_ARG
    lib.ptp_batch_destroy.argtypes = [ctypes.c_void_p]
    assert lib.ptp_batch_destroy(None) == capi.PTP_ERR_ARG


def test_autotune_argument_errors_before_cuda(lib):
    from paper_1810_08218_gb300 import capi

    lib.ptp_autotune.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    p = capi.Params()
    assert lib.ptp_autotune(None, None, ctypes.byref(p), 3, None, None) == capi.PTP_ERR_ARG  # neither target
    assert lib.ptp_autotune(ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.byref(p), 3, None, None) == capi.PTP_ERR_ARG
    assert lib.ptp_autotune(ctypes.c_void_p(8), None, None, 3, None, None) == capi.PTP_ERR_ARG


def test_selftest_argument_errors_before_cuda(lib):
    from paper_1810_08218_gb300 import capi

    lib.ptp_selftest_wait_limit.argtypes = [ctypes.c_int64, ctypes.c_void_p]
    assert lib.ptp_selftest_wait_limit(10, None) == capi.PTP_ERR_ARG
    assert lib.ptp_selftest_wait_limit(10**12, None) == capi.PTP_ERR_ARG
