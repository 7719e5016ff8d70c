"""ctypes declarations of the C-ABI in include/bridge.h.

Loads the in-tree ``libbridge.so`` and fails loudly when it is missing: there
is no CPU or eager fallback for any operation of this package.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_long, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbridge.so")

BRIDGE_OK = 0
BRIDGE_PENDING = 1
BRIDGE_EINVAL = -1
BRIDGE_ENOMEM = -2
BRIDGE_ENOCONV = -3
BRIDGE_EBREAKDOWN = -4
BRIDGE_ETIMEDOUT = -5
BRIDGE_ECUDA = -6
BRIDGE_ESTATE = -7

BRIDGE_F64, BRIDGE_F32, BRIDGE_F16, BRIDGE_BF16 = 0, 1, 2, 3
BRIDGE_METHOD_AUTO, BRIDGE_METHOD_BICGSTAB, BRIDGE_METHOD_CGNR = 0, 1, 2
BRIDGE_WILSON, BRIDGE_CLOVER, BRIDGE_MOBIUS, BRIDGE_STAGGERED = 0, 1, 2, 3
BRIDGE_EVEN, BRIDGE_ODD, BRIDGE_FULL = 0, 1, 2
BRIDGE_APPLY_D, BRIDGE_APPLY_DEO, BRIDGE_APPLY_DOE, BRIDGE_APPLY_DHAT = 0, 1, 2, 3
BRIDGE_NOALLOC_SCRATCH_BYTES = 64 << 20


class bridge_op(ctypes.Structure):
    _fields_ = [
        ("kind", c_int),
        ("kappa", c_double),
        ("csw", c_double),
        ("bc", c_int * 4),
        ("Ls", c_int),
        ("M5", c_double),
        ("b5", c_double),
        ("c5", c_double),
        ("mf", c_double),
        ("mass", c_double),
    ]


class bridge_solver(ctypes.Structure):
    _fields_ = [
        ("tol", c_double),
        ("max_iter", c_int),
        ("inner_prec", c_int),
        ("inner_tol", c_double),
        ("mixed", c_int),
        ("check_every", c_int),
        ("use_graph", c_int),
        ("max_outer", c_int),
        ("method", c_int),
    ]


class bridge_dd_plan(ctypes.Structure):
    _fields_ = [
        ("local_dims", c_int * 4),
        ("t0", c_int),
        ("rank_up", c_int),
        ("rank_down", c_int),
        ("face_sites", c_long),
        ("up_wraps", c_int),
        ("down_wraps", c_int),
        ("canon_offset_sites", c_long),
    ]


class bridge_info(ctypes.Structure):
    _fields_ = [
        ("status", c_int),
        ("outer_iters", c_int),
        ("inner_iters", c_int),
        ("restarts", c_int),
        ("true_rel_residual", c_double),
        ("seconds", c_double),
        ("cgnr_passes", c_int),
    ]


class bridge_mg_params(ctypes.Structure):
    _fields_ = [
        ("block", c_int * 4),
        ("nvec", c_int),
        ("setup_tol", c_double),
        ("setup_steps", c_int),
        ("sap_cycles", c_int),
        ("mr_steps", c_int),
        ("coarse_tol", c_double),
        ("coarse_maxiter", c_int),
        ("coarse_half", c_int),
        ("coarse_eo", c_int),
    ]


BRIDGE_MG_RESTRICT, BRIDGE_MG_PROLONG, BRIDGE_MG_COARSE, BRIDGE_MG_SAP, BRIDGE_MG_CYCLE = 0, 1, 2, 3, 4
BRIDGE_MG_COARSE_HALF, BRIDGE_MG_COARSE_SOLVE = 5, 6


class bridge_kstat(ctypes.Structure):
    _fields_ = [("name", c_char_p), ("launches", c_long), ("bytes", c_double), ("flops", c_double), ("ms", c_double)]


_dp = POINTER(c_double)
_h = c_void_p  # opaque handles

SIGNATURES = {
    "bridge_lattice_create": (c_int, [POINTER(c_int), POINTER(_h)]),
    "bridge_lattice_destroy": (c_int, [_h]),
    "bridge_lattice_stream": (c_void_p, [_h]),
    "bridge_sync": (c_int, [_h]),
    "bridge_gauge_upload": (c_int, [_h, _dp, POINTER(bridge_op)]),
    "bridge_gauge_upload_dev": (c_int, [_h, c_void_p, POINTER(bridge_op)]),
    "bridge_mult_D": (c_int, [_h, POINTER(bridge_op), c_int, _dp, _dp, c_int]),
    "bridge_mult_Deo": (c_int, [_h, POINTER(bridge_op), c_int, c_int, _dp, _dp, c_int]),
    "bridge_mult_Dhat": (c_int, [_h, POINTER(bridge_op), c_int, _dp, _dp, c_int]),
    "bridge_mult_Dhat_dag": (c_int, [_h, POINTER(bridge_op), c_int, _dp, _dp, c_int]),
    "bridge_mult_D_dev": (c_int, [_h, POINTER(bridge_op), c_int, c_void_p, c_void_p, c_int]),
    "bridge_mult_Deo_dev": (c_int, [_h, POINTER(bridge_op), c_int, c_int, c_void_p, c_void_p, c_int]),
    "bridge_mult_Dhat_dev": (c_int, [_h, POINTER(bridge_op), c_int, c_void_p, c_void_p, c_int]),
    "bridge_mult_Dhat_dag_dev": (c_int, [_h, POINTER(bridge_op), c_int, c_void_p, c_void_p, c_int]),
    "bridge_mult_Dhat_noalloc": (c_int, [_h, POINTER(bridge_op), c_int, c_void_p, c_void_p, c_int]),
    "bridge_solve": (c_int, [_h, POINTER(bridge_op), POINTER(bridge_solver), _dp, _dp, c_int, POINTER(bridge_info)]),
    "bridge_solve_dev": (
        c_int,
        [_h, POINTER(bridge_op), POINTER(bridge_solver), c_void_p, c_void_p, c_int, POINTER(bridge_info)],
    ),
    "bridge_solver_defaults": (None, [POINTER(bridge_solver)]),
    "bridge_field_create": (c_int, [_h, c_int, c_int, c_int, POINTER(_h)]),
    "bridge_field_destroy": (c_int, [_h]),
    "bridge_field_import": (c_int, [_h, c_void_p, c_int]),
    "bridge_field_export": (c_int, [_h, c_void_p, c_int]),
    "bridge_apply": (c_int, [_h, POINTER(bridge_op), c_int, _h, _h]),
    "bridge_engine_config": (c_int, [c_size_t, c_int]),
    "bridge_submit": (c_int, [_h, POINTER(bridge_op), POINTER(bridge_solver), _dp, c_int, POINTER(_h)]),
    "bridge_submit_borrowed": (c_int, [_h, POINTER(bridge_op), POINTER(bridge_solver), _dp, c_int, POINTER(_h)]),
    "bridge_mg_defaults": (None, [POINTER(bridge_mg_params)]),
    "bridge_mg_setup": (c_int, [_h, POINTER(bridge_op), POINTER(bridge_mg_params), _dp, POINTER(_h)]),
    "bridge_mg_destroy": (c_int, [_h]),
    "bridge_mg_solve": (c_int, [_h, POINTER(bridge_solver), _dp, _dp, c_int, POINTER(bridge_info)]),
    "bridge_mg_solve_dev": (c_int, [_h, POINTER(bridge_solver), c_void_p, c_void_p, c_int, POINTER(bridge_info)]),
    "bridge_mg_apply": (c_int, [_h, c_int, _dp, _dp]),
    "bridge_mg_coarse_matrix": (c_int, [_h, _dp]),
    "bridge_mg_info": (c_int, [_h, POINTER(c_int), POINTER(c_int)]),
    "bridge_mg_counters": (c_int, [_h, POINTER(c_long), POINTER(c_long)]),
    "bridge_poll": (c_int, [_h, _dp, POINTER(bridge_info)]),
    "bridge_wait": (c_int, [_h, c_int, _dp, POINTER(bridge_info)]),
    "bridge_request_release": (c_int, [_h]),
    "bridge_request_times": (c_int, [_h, _dp, _dp, _dp]),
    "bridge_strerror": (c_char_p, [c_int]),
    "bridge_last_error": (c_char_p, []),
    "bridge_stats": (c_int, [_h, POINTER(bridge_kstat), c_int]),
    "bridge_stats_reset": (c_int, [_h]),
    "bridge_profile": (c_int, [_h, c_int]),
    "bridge_launch_count": (c_long, []),
    "bridge_dd_plan_of": (c_int, [POINTER(c_int), c_int, c_int, POINTER(bridge_dd_plan)]),
    "bridge_dd_create": (c_int, [_h, POINTER(bridge_op), c_int, POINTER(_h)]),
    "bridge_dd_destroy": (c_int, [_h]),
    "bridge_dd_mult_D_dev": (c_int, [_h, c_int, c_void_p, c_void_p, c_int]),
    "bridge_dd_mult_Deo_dev": (c_int, [_h, c_int, c_int, c_void_p, c_void_p, c_int]),
    "bridge_dd_mult_Dhat_dev": (c_int, [_h, c_int, c_void_p, c_void_p, c_int]),
    "bridge_dd_solve_dev": (c_int, [_h, POINTER(bridge_solver), c_void_p, c_void_p, c_int, POINTER(bridge_info)]),
    "bridge_device_alloc_count": (c_long, []),
    "bridge_alu_peak": (c_int, [c_int, _dp]),
    "bridge_tune": (c_int, [_h, POINTER(bridge_op), c_int, c_int]),
    "bridge_tune_table": (c_int, [_h, c_char_p, c_int]),
    "bridge_tune_set": (c_int, [_h, c_char_p, c_int, c_int, c_int]),
    "bridge_debug_neighbours": (c_int, [POINTER(c_int), c_int, c_long, POINTER(c_long), POINTER(c_int)]),
}

_lib = None


def load():
    """Load libbridge.so once and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
            "(there is no CPU fallback)"
        )
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class BridgeError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        detail = lib.bridge_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.bridge_strerror(status).decode()} ({status}): {detail}")
        self.status = status


def check(status: int, where: str) -> int:
    if status < 0:
        raise BridgeError(status, where)
    return status
