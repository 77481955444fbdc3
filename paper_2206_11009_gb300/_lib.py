"""ctypes view of the C ABI in ``include/ot_ipm.h`` (argument marshalling only).

The shared library is ``_build/libotipm.so`` inside this package, built by ``build.py``.
Loading fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libotipm.so")

OT_OK, OT_ERR_ARG, OT_ERR_CUDA, OT_ERR_OOM, OT_ERR_MAXITER, OT_ERR_NUMERIC, OT_ERR_TIMEOUT, \
    OT_ERR_BUF_TOO_SMALL, OT_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = ["OT_OK", "OT_ERR_ARG", "OT_ERR_CUDA", "OT_ERR_OOM", "OT_ERR_MAXITER", "OT_ERR_NUMERIC",
                "OT_ERR_TIMEOUT", "OT_ERR_BUF_TOO_SMALL", "OT_ERR_UNSUPPORTED"]
COST = {"sqeuclid": 0, "euclid": 1, "l1": 2, "linf": 3, "dense": 4}


class OtProblem(ctypes.Structure):
    _fields_ = [("m", c_int32), ("n", c_int32), ("a", c_void_p), ("b", c_void_p), ("cost", c_int32),
                ("src_x", c_void_p), ("src_y", c_void_p), ("dst_x", c_void_p), ("dst_y", c_void_p),
                ("src_w", c_int32), ("dst_w", c_int32), ("C", c_void_p), ("inputs_on_device", c_int32)]


class OtOptions(ctypes.Structure):
    _fields_ = [("tol", c_double), ("feas_l1", c_double), ("cg_tol_pred", c_double), ("cg_tol_corr", c_double),
                ("max_iter", c_int32), ("max_cg", c_int32), ("max_corr", c_int32), ("step_scale", c_double),
                ("precision", c_int32), ("linear_solver", c_int32), ("init_cost", c_double),
                ("rm_mu_frac", c_double), ("rm_p_frac", c_double), ("add_max", c_int32), ("verbose", c_int32),
                ("stream", c_void_p), ("warm_u", c_void_p), ("warm_v", c_void_p), ("warm_count", c_int32),
                ("warm_mode", c_int32), ("warm_i", c_void_p), ("warm_j", c_void_p), ("warm_npairs", c_int64),
                ("new_col_rule", c_int32), ("scan_rows", c_int32), ("dense32_max_n", c_int32),
                ("dense_max_n", c_int32), ("jset_cmax", c_double), ("jset_refresh", c_int32),
                ("multiscale", c_int32), ("ms_tol", c_double), ("precond", c_int32), ("ic_tau", c_double),
                ("tc_update", c_int32), ("direct_cg_tol", c_double)]


class OtPriceOpts(ctypes.Structure):
    _fields_ = [("cost", c_int32), ("scan_rows", c_int32), ("jset_cmax", c_double), ("C", c_void_p)]


class OtIterInfo(ctypes.Structure):
    _fields_ = [("iter", c_int32), ("psi", c_int64), ("mu", c_double), ("crit", c_double),
                ("alpha_p", c_double), ("alpha_s", c_double), ("sigma", c_double), ("ncorr", c_int32),
                ("cg_iters", c_int32), ("direct", c_int32), ("added", c_int64), ("removed", c_int64),
                ("done", c_int32)]


class OtResult(ctypes.Structure):
    _fields_ = [("status", c_int32), ("obj", c_double), ("lower_bound", c_double), ("rel_gap", c_double),
                ("r1_l1", c_double), ("mu", c_double), ("iters", c_int32), ("cg_iters", c_int32),
                ("direct_iters", c_int32), ("psi", c_int64), ("max_fill", c_double), ("seconds", c_double),
                ("warm_added", c_int64), ("warm_restarts", c_int32), ("create_seconds", c_double),
                ("ms_levels", c_int32)]


# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "ot_options_default": (None, [POINTER(OtOptions)]),
    "ot_ipm_create": (c_int32, [POINTER(OtProblem), POINTER(OtOptions), POINTER(c_void_p)]),
    "ot_ipm_step": (c_int32, [c_void_p, POINTER(OtIterInfo)]),
    "ot_ipm_solve": (c_int32, [c_void_p, POINTER(OtResult)]),
    "ot_ipm_get_solution": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, POINTER(c_int64),
                                      c_void_p, c_void_p]),
    "ot_ipm_get_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, POINTER(c_int64),
                                   c_void_p, c_void_p]),
    "ot_ipm_newton_direction": (c_int32, [c_void_p, c_int32, c_double, c_int32, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_int64, POINTER(c_int32)]),
    "ot_ipm_set_state": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p,
                                   c_int32]),
    "ot_ipm_mass_scale": (c_double, [c_void_p]),
    "ot_ipm_ic_apply": (c_int32, [c_void_p, c_double, c_void_p, c_void_p]),
    "ot_ipm_destroy": (None, [c_void_p]),
    "ot_ipm_last_error": (c_char_p, [c_void_p]),
    "ot_last_error": (c_char_p, []),
    "ot_price_topk": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_int64, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p]),
    "ot_price_topk_ex": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_int64, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                   c_void_p, POINTER(OtPriceOpts), c_void_p]),
    "ot_price_topk_noalloc": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p]),
    "ot_kernel_launches": (c_int64, []),
    "ot_abi_struct_sizes": (c_int32, [c_void_p, c_int32]),
    "ot_kernel_timing_enable": (None, [c_int32]),
    "ot_kernel_timing_read": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "ot_ipm_solve_batch": (c_int32, [c_void_p, c_int32, c_void_p, c_int32]),
    "ot_cnn_param_count": (c_int64, [c_int32]),
    "ot_cnn_create": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p]),
    "ot_cnn_get_params": (c_int32, [c_void_p, c_void_p, c_int64]),
    "ot_cnn_forward": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "ot_cnn_loss": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ot_cnn_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ot_cnn_adam": (c_int32, [c_void_p, c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              c_int32]),
    "ot_cnn_last_error": (ctypes.c_char_p, [c_void_p]),
    "ot_cnn_destroy": (None, [c_void_p]),
}

KERNEL_IDS = ["scan_hist", "scan_gather", "recheck", "pcg64", "pcg32", "ldl_numeric", "ldl_solve",
              "d32_factor", "d32_apply", "dcg"]

_lib = None


def load(path: str | None = None):
    """Load (once) and return the library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found at {path}: build it with "
                           "paper_2206_11009_gb300.build.build() (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class OTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        name = STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else str(code)
        super().__init__(f"{name}: {msg}")
        self.code = code


def check(code: int, handle=None):
    if code != OT_OK:
        lib = load()
        msg = lib.ot_ipm_last_error(handle) if handle else lib.ot_last_error()
        raise OTError(code, (msg or b"").decode(errors="replace"))
