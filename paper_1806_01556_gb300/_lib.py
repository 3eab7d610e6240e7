"""ctypes declarations of the libfdas C ABI (include/fdas.h), with the same names.

This module only loads the shared library and declares argument types. If libfdas.so is
missing it raises: the package has no CPU or fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfdas.so")

FDAS_OK = 0
FDAS_ERR_INVALID_ARG = -1
FDAS_ERR_UNSUPPORTED = -2
FDAS_ERR_WORKSPACE = -3
FDAS_ERR_CUDA = -4
FDAS_ERR_TIMEOUT = -5
FDAS_DEV_WAIT_TIMEOUT = 1

FDAS_FP32, FDAS_BF16X3, FDAS_FP16S = 0, 1, 2
FDAS_INDEX_FUNDAMENTAL, FDAS_INDEX_HIGHEST = 0, 1
FDAS_MAX_N = 1 << 24
FDAS_RAW_CAP = 16384
FDAS_MAX_CAND_CAP = 4096
FDAS_MAX_HARM = 16
FDAS_NOALLOC_SCRATCH_BYTES = 8 * 8 * (FDAS_RAW_CAP + 4)
FDAS_MAX_BATCH = 256


class fdas_params(C.Structure):
    _fields_ = [
        ("n_temp", C.c_int32),
        ("z_min", C.c_int32),
        ("z_step", C.c_int32),
        ("n_tap", C.c_int32),
        ("fft_len", C.c_int32),
        ("n_harm", C.c_int32),
        ("harm_mask", C.c_uint32),
        ("cand_cap", C.c_int32),
        ("precision", C.c_int32),
        ("harm_index", C.c_int32),
    ]


class fdas_launch_config(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("templates_per_item", C.c_int32)]


class fdas_batch_item(C.Structure):
    _fields_ = [
        ("d_spec", C.c_void_p),
        ("n", C.c_uint64),
        ("d_plane", C.c_void_p),
        ("ld", C.c_uint64),
        ("d_cands", C.c_void_p),
        ("d_counts", C.c_void_p),
        ("d_peaks", C.c_void_p),
    ]


class fdas_cand(C.Structure):
    _fields_ = [("power", C.c_float), ("j", C.c_uint32), ("i", C.c_int16), ("k", C.c_uint8), ("pad", C.c_uint8)]


class fdas_result(C.Structure):
    _fields_ = [
        ("id", C.c_uint64),
        ("n", C.c_uint64),
        ("status", C.c_int32),
        ("pad", C.c_int32),
        ("submit_s", C.c_double),
        ("admit_s", C.c_double),
        ("done_s", C.c_double),
        ("counts", C.c_uint32 * 16),
        ("peaks", fdas_cand * 16),
    ]


P = C.POINTER(fdas_params)
VP = C.c_void_p
SZ = C.c_size_t

# name -> (restype, argtypes); the same list as include/fdas.h
SIGNATURES = {
    "fdas_default_params": (None, [P]),
    "fdas_check_params": (C.c_int, [P]),
    "fdas_status_string": (C.c_char_p, [C.c_int]),
    "fdas_last_error": (C.c_char_p, []),
    "fdas_device_status": (C.c_int, [C.POINTER(C.c_uint32), C.c_int]),
    "fdas_set_device_status": (C.c_int, [C.c_uint32]),
    "fdas_measure_fp32_peak": (C.c_int, [C.c_float, C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    "fdas_check_wait_timeout": (C.c_int, [C.POINTER(C.c_uint32)]),
    "fdas_templates_bytes": (SZ, [P]),
    "fdas_plane_bytes": (SZ, [P, SZ, SZ]),
    "fdas_workspace_bytes": (SZ, [P, SZ]),
    "fdas_default_thresholds": (C.c_int, [P, C.c_double, C.c_int, VP]),
    "fdas_make_templates": (C.c_int, [P, VP, VP]),
    "fdas_convolve": (C.c_int, [P, VP, SZ, VP, VP, SZ, VP]),
    "fdas_convolve_cfg": (C.c_int, [P, VP, SZ, VP, VP, SZ, VP, VP]),
    "fdas_harmonic_sum": (C.c_int, [P, VP, SZ, SZ, VP, VP, VP, VP, VP, SZ, VP]),
    "fdas_search": (C.c_int, [P, VP, SZ, VP, VP, SZ, VP, VP, VP, VP, VP, SZ, VP]),
    "fdas_search_convolve": (C.c_int, [P, VP, SZ, VP, VP, SZ, VP, VP, SZ, VP]),
    "fdas_search_harmonic": (C.c_int, [P, VP, SZ, SZ, VP, VP, VP, VP, VP, SZ, VP]),
    "fdas_search_host": (C.c_int, [P, VP, SZ, VP, VP, VP, SZ, VP, VP, VP, VP, VP, VP, VP, VP, SZ, VP]),
    "fdas_search_host_async": (C.c_int, [P, VP, SZ, VP, VP, VP, SZ, VP, VP, VP, VP, VP, VP, VP, VP, SZ, VP]),
    "fdas_harmonic_sum_noalloc": (C.c_int, [P, VP, SZ, SZ, VP, VP, VP, VP, VP]),
    "fdas_batch_workspace_bytes": (SZ, [P, C.c_int]),
    "fdas_search_batch": (C.c_int, [P, VP, C.c_int, VP, VP, VP, SZ, VP, VP]),
    "fdas_harmonic_sum_batch": (C.c_int, [P, VP, C.c_int, VP, VP, SZ, VP]),
    "fdas_batch_plan_create": (C.c_int, [P, VP, C.c_int, VP, VP, VP, SZ, C.POINTER(C.c_void_p)]),
    "fdas_batch_plan_tune": (C.c_int, [VP, VP, VP, C.POINTER(C.c_float)]),
    "fdas_batch_plan_launch": (C.c_int, [VP, VP]),
    "fdas_batch_plan_destroy": (None, [VP]),
    "fdas_server_create": (C.c_int, [P, SZ, C.c_int, C.POINTER(C.c_void_p)]),
    "fdas_server_request_bytes": (SZ, [P, C.c_uint64]),
    "fdas_server_submit": (C.c_int, [VP, VP, C.c_uint64, C.c_uint64, VP]),
    "fdas_server_poll": (C.c_int, [VP, VP, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "fdas_server_stats": (None, [VP, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fdas_server_destroy": (None, [VP]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libfdas.so once and declare every entry point. Raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"libfdas.so not found at {path}; build it with `python -m paper_1806_01556_gb300.build` "
            "(there is no fallback path)"
        )
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
