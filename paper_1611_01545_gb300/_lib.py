"""ctypes binding of libpm.so (include/pm.h): structures and prototypes only.

The library is built in-tree by ``paper_1611_01545_gb300.build``; importing
this module fails loudly if it is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpm.so")

PM_OK = 0
PM_ERR_ARG = 1
PM_ERR_CONFIG = 2
PM_ERR_CUDA = 3
PM_ERR_CORRUPT = 4
PM_ERR_OVERFLOW = 5
PM_ERR_RANGE = 6
PM_ERR_TIMEOUT = 7

ERROR_NAMES = {0: "PM_OK", 1: "PM_ERR_ARG", 2: "PM_ERR_CONFIG", 3: "PM_ERR_CUDA", 4: "PM_ERR_CORRUPT",
               5: "PM_ERR_OVERFLOW", 6: "PM_ERR_RANGE", 7: "PM_ERR_TIMEOUT"}


class pm_config_t(ctypes.Structure):
    _fields_ = [("n_fine", ctypes.c_int32), ("coarse_ratio", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("buffer", ctypes.c_int32), ("cmp_ratio", ctypes.c_int32), ("vel_bits", ctypes.c_int32),
                ("deposit_mode", ctypes.c_int32), ("tile_batch", ctypes.c_int32), ("vmax_mode", ctypes.c_int32),
                ("pp", ctypes.c_int32), ("G", ctypes.c_double),
                ("mass", ctypes.c_double * 2), ("count", ctypes.c_int64 * 2), ("r_split", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("r_soft", ctypes.c_double)]


class pm_tuning_t(ctypes.Structure):
    _fields_ = [("deposit_block", ctypes.c_int32 * 3), ("deposit_persistent", ctypes.c_int32),
                ("kick_block", ctypes.c_int32 * 3), ("kick_window", ctypes.c_int32),
                ("kick_persistent", ctypes.c_int32), ("tile_batch", ctypes.c_int32)]


class pm_particles_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("v", ctypes.c_void_p)]


class pm_codes_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cnt", ctypes.c_void_p), ("esc", ctypes.c_void_p),
                ("esc_cap", ctypes.c_int64), ("n_esc", ctypes.c_void_p), ("pos", ctypes.c_void_p),
                ("vel", ctypes.c_void_p), ("vmax", ctypes.c_void_p)]


EXPORTED = ["pm_init", "pm_destroy", "pm_geometry", "pm_decompress", "pm_compress", "pm_deposit",
            "pm_deposit_weights", "pm_deposit_fixed", "pm_deposit_codes", "pm_tile_density", "pm_solve", "pm_solve_fixed", "pm_interpolate",
            "pm_kick_drift", "pm_step", "pm_step_host", "pm_check", "pm_last_error", "pm_set_timing", "pm_set_graphs",
            "pm_get_tuning", "pm_set_tuning", "pm_autotune", "pm_pp_accel",
            "pm_checkpoint_begin", "pm_checkpoint_fence", "pm_checkpoint_wait", "pm_pack_codes", "pm_unpack_codes",
            "pm_step_packed", "pm_step_packed_async", "pm_restrict",
            "pm_stage_times", "pm_serialize", "pm_deserialize", "pm_error_string", "pm_launch_count",
            "pm_decompress_noalloc", "pm_deposit_adjoint", "pm_solve_adjoint", "pm_interpolate_adjoint",
            "pm_step_adjoint", "pm_step_adjoint_acc", "pm_wait_probe"]

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_PROTOS = {
    "pm_init": (ctypes.c_int, [ctypes.POINTER(pm_config_t), ctypes.POINTER(_P)]),
    "pm_destroy": (ctypes.c_int, [_P]),
    "pm_geometry": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                   ctypes.POINTER(_I64)]),
    "pm_decompress": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(pm_codes_t), _P, _P, _P]),
    "pm_compress": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(pm_codes_t), _P]),
    "pm_deposit": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, _P, _P, _P]),
    "pm_deposit_weights": (ctypes.c_int, [_P, _P, _I64, _P, ctypes.c_int32, _P, _P]),
    "pm_deposit_fixed": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, _P, _P, _P]),
    "pm_deposit_codes": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), _P, _P, _P]),
    "pm_tile_density": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "pm_solve": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "pm_solve_fixed": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "pm_interpolate": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P]),
    "pm_kick_drift": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P, _D, _D, _P]),
    "pm_step": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), _D, _D, _P]),
    "pm_step_host": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), _D, _D, _P]),
    "pm_check": (ctypes.c_int, [_P, _P]),
    "pm_wait_probe": (ctypes.c_int, [_P, _I64, _P]),
    "pm_last_error": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "pm_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "pm_set_graphs": (ctypes.c_int, [_P, ctypes.c_int]),
    "pm_pp_accel": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), _P, _P]),
    "pm_checkpoint_begin": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), _P]),
    "pm_checkpoint_fence": (ctypes.c_int, [_P, _P]),
    "pm_checkpoint_wait": (ctypes.c_int, [_P]),
    "pm_restrict": (ctypes.c_int, [_P, _P, _P, _P]),
    "pm_pack_codes": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), _P]),
    "pm_unpack_codes": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), _P]),
    "pm_step_packed": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), _D, _D, _P]),
    "pm_step_packed_async": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), _D, _D,
                                            _P]),
    "pm_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(pm_tuning_t)]),
    "pm_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(pm_tuning_t)]),
    "pm_autotune": (ctypes.c_int, [_P, ctypes.POINTER(pm_codes_t), ctypes.POINTER(pm_codes_t), ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int32, _P, ctypes.POINTER(pm_tuning_t)]),
    "pm_stage_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.c_char_p, ctypes.c_size_t]),
    "pm_serialize": (ctypes.c_int, [ctypes.POINTER(pm_codes_t), ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t,
                                    ctypes.POINTER(ctypes.c_size_t)]),
    "pm_deserialize": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(pm_codes_t)]),
    "pm_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pm_launch_count": (ctypes.c_int64, []),
    "pm_deposit_adjoint": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, _P, _P, _P]),
    "pm_solve_adjoint": (ctypes.c_int, [_P, _P, _P, _P]),
    "pm_interpolate_adjoint": (ctypes.c_int, [_P, _P, _I64, _P, _D, _D, _P, _P, _P, _P]),
    "pm_step_adjoint": (ctypes.c_int, [_P, ctypes.POINTER(pm_particles_t), ctypes.POINTER(pm_particles_t), _D, _D,
                                       _P]),
    "pm_step_adjoint_acc": (ctypes.c_int, [_P, ctypes.POINTER(pm_particles_t), ctypes.POINTER(pm_particles_t), _P,
                                           _D, _D, _P]),
    "pm_decompress_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(pm_codes_t), _P, _P, _P]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpm.so and declare every prototype; raises if the library is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpm.so not found at {path}: build it with "
                          "`python -m paper_1611_01545_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
