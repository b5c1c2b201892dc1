"""ctypes declarations of the C ABI in include/tdse.h (argument marshalling only).

The shared library is built in-tree (``python -m paper_2001_06113_gb300.build``
or ``__graft_entry__.build()``).  Loading fails loudly when it is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtdse_gb300.so")

TDSE_OK = 0
STATUS_NAMES = {0: "TDSE_OK", -1: "TDSE_EINVAL", -2: "TDSE_ENOMEM", -3: "TDSE_ECUDA", -4: "TDSE_ETIMEOUT",
                -5: "TDSE_ENONFINITE", -6: "TDSE_ESTATE", -7: "TDSE_EUNSUPPORTED"}
PERIODIC, FREE = 0, 1
FP64, MIXED = 0, 1
HOST, DEVICE = 0, 1
TDSE_V_SEPARABLE, TDSE_V_TABLE, TDSE_V_TABLE_SHARED = 0, 1, 2
TDSE_ESTATE = -6
PATH_AUTO, PATH_PASSES, PATH_CLUSTER = 0, 1, 2

# Every symbol include/tdse.h declares (checked by the CPU test suite).
EXPORTS = [
    "tdse_create", "tdse_workspace_bytes", "tdse_bind_workspace", "tdse_set_potential",
    "tdse_set_vector_potential", "tdse_set_pulse", "tdse_set_initial", "tdse_set_initial_batch", "tdse_step", "tdse_solve_to",
    "tdse_read_u", "tdse_check_finite", "tdse_step_index", "tdse_time", "tdse_adams_weights",
    "tdse_last_error", "tdse_destroy", "tdse_modes_to_grid_2d_noalloc", "tdse_read_modes", "tdse_free_rule",
    "tdse_free_choose_H", "tdse_free_choose_H_prec", "tdse_potential_times", "tdse_set_potential_table", "tdse_batch_create", "tdse_batch_tune", "tdse_batch_set_mode", "tdse_batch_step", "tdse_batch_describe",
    "tdse_batch_last_error", "tdse_batch_destroy", "tdse_set_residual_check", "tdse_residual_report",
    "tdse_save", "tdse_load", "tdse_set_step_path", "tdse_step_path", "tdse_describe_steps", "tdse_set_step_groups", "tdse_free_cheb_terms",
    "tdse_set_shape_1d", "tdse_shape_1d",
]
NOALLOC_MAX_POINTS = 524288


class TdseConfig(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("n", ctypes.c_int * 2),
        ("batch", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("nsteps", ctypes.c_int),
        ("order", ctypes.c_int),
        ("startup_steps", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("nu", ctypes.c_int * 2),
        ("alpert_p", ctypes.c_int),
        ("gauss_q", ctypes.c_int),
        ("n_r", ctypes.c_int),
        ("H", ctypes.c_double),
        ("potential", ctypes.c_int),
        ("n_z", ctypes.c_int),
        ("c_transform", ctypes.c_int),
        ("nu_z", ctypes.c_int),
        ("layout_1d", ctypes.c_int),
    ]


FIELD_FN = ctypes.CFUNCTYPE(None, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


class TdseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = _LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libtdse_gb300.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, ip, dp, cd = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double
    sig = {
        "tdse_create": ([ctypes.POINTER(TdseConfig), ctypes.POINTER(vp)], ip),
        "tdse_workspace_bytes": ([vp], ctypes.c_size_t),
        "tdse_bind_workspace": ([vp, vp, ctypes.c_size_t, vp], ip),
        "tdse_set_potential": ([vp, ip, vp, vp, ip, vp], ip),
        "tdse_set_vector_potential": ([vp, ip, FIELD_FN, vp, vp], ip),
        "tdse_set_pulse": ([vp, ip, cd, cd, cd, dp, vp], ip),
        "tdse_set_initial": ([vp, ip, vp, ip, vp], ip),
        "tdse_set_initial_batch": ([vp, vp, ip, vp], ip),
        "tdse_step": ([vp, ip, vp], ip),
        "tdse_solve_to": ([vp, cd, vp], ip),
        "tdse_read_u": ([vp, ip, vp, ip, vp], ip),
        "tdse_check_finite": ([vp, vp], ip),
        "tdse_step_index": ([vp], ip),
        "tdse_time": ([vp], cd),
        "tdse_adams_weights": ([ip, dp], ip),
        "tdse_last_error": ([vp], ctypes.c_char_p),
        "tdse_destroy": ([vp], None),
        "tdse_modes_to_grid_2d_noalloc": ([vp, vp, ip, ip, ip, vp], ip),
        "tdse_read_modes": ([vp, ip, vp, ip, vp], ip),
        "tdse_free_rule": ([vp, ip, ctypes.POINTER(ip), dp, dp], ip),
        "tdse_free_choose_H": ([cd, cd, cd, ip, dp], ip),
        "tdse_free_choose_H_prec": ([cd, cd, cd, ip, ip, dp], ip),
        "tdse_batch_create": ([ctypes.POINTER(vp), ip, ctypes.POINTER(vp)], ip),
        "tdse_batch_tune": ([vp, ip, vp], ip),
        "tdse_batch_set_mode": ([vp, ip], ip),
        "tdse_batch_step": ([vp, ip, vp], ip),
        "tdse_batch_describe": ([vp, ctypes.c_char_p, ctypes.c_size_t], ip),
        "tdse_batch_last_error": ([vp], ctypes.c_char_p),
        "tdse_batch_destroy": ([vp], None),
        "tdse_set_residual_check": ([vp, ip, cd], ip),
        "tdse_residual_report": ([vp, dp, ctypes.POINTER(ip), ctypes.POINTER(ip), vp], ip),
        "tdse_save": ([vp, vp, ctypes.POINTER(ctypes.c_size_t), vp], ip),
        "tdse_potential_times": ([vp, dp], ip),
        "tdse_set_potential_table": ([vp, ip, vp, ip, vp], ip),
        "tdse_load": ([vp, vp, ctypes.c_size_t, vp], ip),
        "tdse_set_step_path": ([vp, ip], ip),
        "tdse_step_path": ([vp], ip),
        "tdse_describe_steps": ([vp, ctypes.c_char_p, ctypes.c_size_t], ip),
        "tdse_set_step_groups": ([vp, ip], ip),
        "tdse_set_shape_1d": ([vp, ip], ip),
        "tdse_shape_1d": ([vp], ip),
        "tdse_free_cheb_terms": ([vp, ip], ip),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib
