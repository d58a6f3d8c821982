"""ctypes loader for libwpcd.so (the C ABI of include/wpcd.h).

The library is built in place by ``paper_2106_00454_gb300.build.build()``.
There is no fallback: if the shared library is missing or fails to load,
every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libwpcd.so")

# Every entry point declared in include/wpcd.h.
EXPORTED = [
    "wpcd_create", "wpcd_destroy", "wpcd_strerror", "wpcd_set_option", "wpcd_sync", "wpcd_bytes_in_use",
    "wpcd_mesh", "wpcd_mesh_get", "wpcd_project", "wpcd_project_prec", "wpcd_vset_get", "wpcd_vset_info", "wpcd_diag",
    "wpcd_diag_status", "wpcd_eig_get", "wpcd_tmatrix", "wpcd_observables", "wpcd_observables_res", "wpcd_solve", "wpcd_solve_host",
    "wpcd_release", "wpcd_kernel_launches", "wpcd_profile", "wpcd_profile_read",
    "wpcd_channel_solve_noalloc", "wpcd_serve_start", "wpcd_serve_stop", "wpcd_submit", "wpcd_poll", "wpcd_wait",
    "wpcd_release_result", "wpcd_serve_stats", "wpcd_batched_dgemm", "wpcd_tuning", "wpcd_mi_prepare",
    "wpcd_mi_solve", "wpcd_saclay", "wpcd_graph_stats", "wpcd_device_log", "wpcd_set_interp_point",
]


class wpcd_channel(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("J", ctypes.c_int), ("l", ctypes.c_int), ("lp", ctypes.c_int),
                ("coupled", ctypes.c_int), ("tz", ctypes.c_int)]


class wpcd_request(ctypes.Structure):
    _fields_ = [("coeffs", ctypes.POINTER(ctypes.c_double)), ("n_terms", ctypes.c_int),
                ("e_lab", ctypes.POINTER(ctypes.c_double)), ("n_E", ctypes.c_int), ("n_wp", ctypes.c_int),
                ("prec", ctypes.c_int)]


class wpcd_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n_E", ctypes.c_int), ("n_ch", ctypes.c_int),
                ("delta", ctypes.POINTER(ctypes.c_double)), ("sigma", ctypes.POINTER(ctypes.c_double)),
                ("T", ctypes.POINTER(ctypes.c_double)), ("latency_us", ctypes.c_double)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_ip = ctypes.POINTER(ctypes.c_int)
_sz = ctypes.c_size_t
_SIG = {
    "wpcd_create": (_i, [ctypes.POINTER(_vp), _i, _sz, _vp]),
    "wpcd_destroy": (None, [_vp]),
    "wpcd_strerror": (ctypes.c_char_p, [_i]),
    "wpcd_set_option": (_i, [_vp, _i, _i]),
    "wpcd_set_interp_point": (_i, [_vp, _d]),
    "wpcd_sync": (_i, [_vp]),
    "wpcd_bytes_in_use": (_sz, [_vp]),
    "wpcd_mesh": (_i, [_vp, _i, _i, _d, _d, _d, _i, _i, _ip]),
    "wpcd_mesh_get": (_i, [_vp, _i, _vp, _vp, _vp]),
    "wpcd_project": (_i, [_vp, _ip, ctypes.POINTER(wpcd_channel), _i, _i, _vp, _i, _vp, _i, _ip]),
    "wpcd_project_prec": (_i, [_vp, _ip, ctypes.POINTER(wpcd_channel), _i, _i, _vp, _i, _vp, _i, _i, _ip]),
    "wpcd_vset_get": (_i, [_vp, _i, _i, _vp]),
    "wpcd_vset_info": (_i, [_vp, _i, _ip, _ip, _i, _ip]),
    "wpcd_diag": (_i, [_vp, _i, _vp, _i, _i, _ip]),
    "wpcd_diag_status": (_i, [_vp, _i, _vp]),
    "wpcd_eig_get": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "wpcd_tmatrix": (_i, [_vp, _i, _vp, _i, _i, _vp]),
    "wpcd_observables": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "wpcd_observables_res": (_i, [_vp, _i, _vp, _i, _i, _vp, _vp]),
    "wpcd_saclay": (_i, [_vp, _vp, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _vp]),
    "wpcd_mi_prepare": (_i, [_vp, _vp, _i, _i, _vp, _i, _i, _i, ctypes.c_double, _vp]),
    "wpcd_mi_solve": (_i, [_vp, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _vp, _vp, _vp]),
    "wpcd_solve": (_i, [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp, _vp, _vp]),
    "wpcd_solve_host": (_i, [_vp, _i, _vp, _i, _vp, _i, _i, _i, _vp, _vp, _vp]),
    "wpcd_release": (_i, [_vp, _i]),
    "wpcd_kernel_launches": (ctypes.c_ulonglong, [_vp]),
    "wpcd_profile": (_i, [_vp, _i]),
    "wpcd_profile_read": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)]),
    "wpcd_channel_solve_noalloc": (_i, [_i, _i, _d, _d, _d, _i, _i, wpcd_channel, _vp, _i, _vp, _i, _vp, _i, _vp,
                                        _vp, _vp, _vp]),
    "wpcd_serve_start": (_i, [_vp, ctypes.POINTER(wpcd_channel), _i, _i, _vp, _i, _i, _ip, _i, _i, _i, _i]),
    "wpcd_serve_stop": (_i, [_vp]),
    "wpcd_submit": (_i, [_vp, ctypes.POINTER(wpcd_request), ctypes.POINTER(ctypes.c_uint64)]),
    "wpcd_poll": (_i, [_vp, ctypes.c_uint64, ctypes.POINTER(wpcd_result)]),
    "wpcd_wait": (_i, [_vp, ctypes.c_uint64, _i, ctypes.POINTER(wpcd_result)]),
    "wpcd_release_result": (None, [_vp, ctypes.c_uint64]),
    "wpcd_batched_dgemm": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _i]),
    "wpcd_tuning": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "wpcd_serve_stats": (_i, [_vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong),
                              ctypes.POINTER(ctypes.c_ulonglong)]),
    "wpcd_graph_stats": (_i, [_vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong),
                              ctypes.POINTER(ctypes.c_int)]),
    "wpcd_device_log": (_i, [_vp, _vp, _vp, _i]),
}

_lock = threading.Lock()
_lib = None


def load():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2106_00454_gb300.build.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIG.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    """Names from EXPORTED that the shared library exports (no device needed)."""
    lib = load()
    return [n for n in EXPORTED if hasattr(lib, n)]
