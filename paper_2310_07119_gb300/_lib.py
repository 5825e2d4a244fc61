"""ctypes declarations of the C ABI in include/twa.h (argument marshalling only).

Every step of the method runs in libtwa.so; if the library is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtwa.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "twa.h")

TWA_OK, TWA_EINVAL, TWA_ENOMEM, TWA_ECUDA, TWA_ETIMEOUT, TWA_ENONFINITE = 0, -1, -2, -3, -4, -5
TWA_F32, TWA_F64_PLAIN = 0, 1
TWA_NSCALARS = 8
TWA_OBS_OF_MEAN, TWA_OBS_MODES, TWA_OBS_FP32 = 1, 2, 4
TWA_BATCH_SERIAL, TWA_BATCH_FORK, TWA_BATCH_PERSISTENT = 0, 1, 2
SCALAR_NAMES = ("Q", "corr", "mass", "mass_cl", "nonfinite", "nk_sum", "drho_l2", "rhocl_l2")
# Pass kinds of the FP32 pipelines, in the library's numbering (profiler ops).
PASS_NAMES = ("drift", "kick_drift", "kick_drift_vinv", "drift_rho", "rho_fwd", "fwd", "fwd_mul_inv", "inv",
              "kick_vinv", "kick_fwd_out", "steps_1d", "mul_inv", "plane_kick_drift", "plane_poisson")
TWA_PROF_NOPS = len(PASS_NAMES)


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("hbar_m", ctypes.c_double), ("C", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_tot", ctypes.c_double), ("noise_conv", ctypes.c_int), ("precision", ctypes.c_int),
                ("want_modes", ctypes.c_int)]


class MomentsOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("rho_mean", "psi_mean", "rho_cl", "nk_mean", "nk_var", "scalars",
                                               "nk_cl")]


class FnoConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("grid", "width", "modes", "layers", "c_in", "c_out")]


_P = ctypes.c_void_p
_SIGS = {
    "twa_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Grid), ctypes.POINTER(Params), ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int)]),
    "twa_destroy": (ctypes.c_int, [_P]),
    "twa_batch_elems": (ctypes.c_size_t, [_P]),
    "twa_sample": (ctypes.c_int, [_P, _P, ctypes.c_uint64, _P, _P]),
    "twa_step_batch": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "twa_moments": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(MomentsOut), _P]),
    "twa_run": (ctypes.c_int, [_P, _P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "twa_advance": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "twa_phase_moments": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "twa_particles_set": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "twa_particles_get": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "twa_advance_adaptive": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P,
                                            ctypes.POINTER(ctypes.c_double), _P]),
    "twa_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "twa_profile_read": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "twa_sync_status": (ctypes.c_int, [_P, _P]),
    "twa_set_batch_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    "twa_get_batch_mode": (ctypes.c_int, [_P]),
    "twa_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_double]),
    "twa_debug_stall_next_batch": (ctypes.c_int, [_P]),
    "twa_debug_stall_next_tma": (ctypes.c_int, [_P]),
    "twa_last_error": (ctypes.c_char_p, [_P]),
    "twa_autotune": (ctypes.c_int, [_P, _P, ctypes.c_char_p, _P]),
    "twa_last_launch_count": (ctypes.c_longlong, [_P]),
    "twa_poisson_multiplier": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "twa_observable_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int]),
    "twa_observable_eval": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "twa_observable_destroy": (ctypes.c_int, [_P]),
    "twa_fno_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(FnoConfig), ctypes.c_uint64]),
    "twa_fno_destroy": (ctypes.c_int, [_P]),
    "twa_fno_num_params": (ctypes.c_longlong, [_P]),
    "twa_fno_set_params": (ctypes.c_int, [_P, _P, _P]),
    "twa_fno_get_params": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "twa_fno_forward": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "twa_fno_backward": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    "twa_fno_zero_grad": (ctypes.c_int, [_P, _P]),
    "twa_fno_adamw": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, _P]),
    "twa_fno_mse": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P, _P, _P]),
    "twa_fno_last_error": (ctypes.c_char_p, [_P]),
    "twa_fno_features": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P, _P, _P]),
    "twa_fno_set_tensor_cores": (ctypes.c_int, [_P, ctypes.c_int]),
    "twa_fno_tensor_core_shapes": (ctypes.c_int, [_P]),
    "twa_fno_sync_status": (ctypes.c_int, [_P, _P]),
    "twa_tc_gemm": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, _P, ctypes.c_int,
                                   ctypes.c_int, _P, ctypes.c_longlong, ctypes.c_int, _P, _P]),
}

_lib = None


def declared_symbols():
    """Function names declared in include/twa.h (parsed from the header text)."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(twa_[a-z_0-9]+)\s*\(", txt, re.M)))


def load():
    """Load libtwa.so and declare its signatures (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
