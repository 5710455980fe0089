"""ctypes loader for libpbng.so (the C ABI of include/pbng.h).

Argument marshalling only: every call goes straight to the C entry point of
the same name.  The library must have been built (``build.py``); there is no
fallback implementation, so a missing library is a hard error.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpbng.so")

PBNG_OK = 0
STATUS_NAMES = {
    0: "PBNG_OK", 1: "PBNG_EINVAL", 2: "PBNG_ENOMEM", 3: "PBNG_ECUDA",
    4: "PBNG_EDEGENERATE", 5: "PBNG_EDIVERGED", 6: "PBNG_ETIMEOUT", 7: "PBNG_ENOTCONVERGED",
}

ACCEL = {"none": 0, "chebyshev": 1, "sor": 2, "cg": 3}
PRECISION = {"fp32": 0, "compensated": 1, "extended": 2, "auto": 3}
MODEL = {"corotated": 0, "neohookean": 1, "stable_neohookean": 2}
ORDER = {"forward": 0, "symmetric": 1}


class PbngParams(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("accel", ctypes.c_int32),
        ("omega", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("step", ctypes.c_double),
        ("skip_tol", ctypes.c_double),
        ("residual_every", ctypes.c_int32),
        ("resume", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("kernel_path", ctypes.c_int32),
        ("colour_order", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]


class PbngProfile(ctypes.Structure):
    _fields_ = [
        ("colour_pass_launches", ctypes.c_int64),
        ("colour_pass_ms", ctypes.c_double),
        ("accel_launches", ctypes.c_int64),
        ("accel_ms", ctypes.c_double),
        ("residual_launches", ctypes.c_int64),
        ("residual_ms", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
        ("free_vertices", ctypes.c_int64),
        ("incidences", ctypes.c_int64),
        ("ncolours", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("colour_ms", ctypes.c_double),
        ("layout_ms", ctypes.c_double),
    ]


MAX_COLOURS = 64      # PBNG_MAX_COLOURS
MAX_CTAS_PER_SM = 2   # PBNG_MAX_CTAS_PER_SM


class PbngSchedule(ctypes.Structure):
    _fields_ = [
        ("ncolours", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32 * MAX_COLOURS),
        ("blocked", ctypes.c_int32 * MAX_COLOURS),
        ("balanced", ctypes.c_int32 * MAX_COLOURS),
        ("default_ms_per_sweep", ctypes.c_double),
        ("tuned_ms_per_sweep", ctypes.c_double),
        ("candidates", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


MAX_SOLVE_EVENTS = 16  # PBNG_MAX_SOLVE_EVENTS


class PbngSolveInfo(ctypes.Structure):
    _fields_ = [
        ("rho", ctypes.c_double),
        ("plain_rate", ctypes.c_double),
        ("estimate_sweeps", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("raises", ctypes.c_int32),
        ("extended_from", ctypes.c_int32),
        ("nevents", ctypes.c_int32),
        ("event_sweep", ctypes.c_int32 * MAX_SOLVE_EVENTS),
        ("event_rho", ctypes.c_double * MAX_SOLVE_EVENTS),
    ]


class PbngNewtonInfo(ctypes.Structure):
    _fields_ = [
        ("newton_iterations", ctypes.c_int32),
        ("cg_iterations", ctypes.c_int32),
        ("line_search_halvings", ctypes.c_int32),
        ("fallbacks", ctypes.c_int32),
        ("rel_residual", ctypes.c_double),
    ]


class PbngError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); every function include/pbng.h declares
SIGNATURES = {
    "pbng_default_params": (None, [ctypes.POINTER(PbngParams)]),
    "pbng_create_mesh": (_I32, [_PD, _I32, _PI, _I32, _PD, _PD, _PI, _P, ctypes.POINTER(_P)]),
    "pbng_set_constraints": (_I32, [_P, _PI, _PD, _I32, _PI, _PD, _PD, _I32, _PD, _D, _PD, _PD]),
    "pbng_set_material": (_I32, [_P, _PD, _PD]),
    "pbng_set_body_accel": (_I32, [_P, _PD, _PD]),
    "pbng_get_colouring": (_I32, [_P, _PI, _PI]),
    "pbng_adjoint": (_I32, [_P, _P, _P, _P, _P, _D, _I32, ctypes.POINTER(PbngParams), _PI, _PD]),
    "pbng_sweep": (_I32, [_P, _P, _I32, ctypes.POINTER(PbngParams), _PD]),
    "pbng_sweep_host": (_I32, [_P, _P, _I32, ctypes.POINTER(PbngParams), _PD]),
    "pbng_solve": (_I32, [_P, _P, _D, _I32, ctypes.POINTER(PbngParams), _PI, _PD]),
    "pbng_residual": (_I32, [_P, _P, _PD]),
    "pbng_get_state": (_I32, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "pbng_set_state": (_I32, [_P, _P, ctypes.c_size_t]),
    "pbng_residual_noalloc": (_I32, [_P, _P, _PD]),
    "pbng_set_profiling": (_I32, [_P, _I32]),
    "pbng_test_set_copy_shortfall": (_I32, [_P, _I32]),
    "pbng_get_profile": (_I32, [_P, ctypes.POINTER(PbngProfile)]),
    "pbng_set_schedule": (_I32, [_P, ctypes.POINTER(PbngParams), ctypes.POINTER(PbngSchedule)]),
    "pbng_get_schedule": (_I32, [_P, ctypes.POINTER(PbngSchedule)]),
    "pbng_autotune": (_I32, [_P, _P, ctypes.POINTER(PbngParams), _I32, ctypes.POINTER(PbngSchedule)]),
    "pbng_get_solve_info": (_I32, [_P, ctypes.POINTER(PbngSolveInfo)]),
    "pbng_measure_fp32_peak": (_I32, [_P, _PD]),
    "pbng_set_inertia": (_I32, [_P, _D, _PD]),
    "pbng_set_weak_constraints": (_I32, [_P, _I32, _PI, _PD, _PD, _PD, _PD, _I32]),
    "pbng_step": (_I32, [_P, _P, _P, _I32, _D, ctypes.POINTER(PbngParams), _PI, _PD]),
    "pbng_set_dirichlet_targets": (_I32, [_P, _PD]),
    "pbng_force": (_I32, [_P, _P, ctypes.POINTER(PbngParams), _P]),
    "pbng_hessian_apply": (_I32, [_P, _P, _P, ctypes.POINTER(PbngParams), _P]),
    "pbng_newton_cg": (_I32, [_P, _P, _D, _I32, _I32, _D, ctypes.POINTER(PbngParams),
                              ctypes.POINTER(PbngNewtonInfo)]),
    "pbng_num_components": (_I32, [_P]),
    "pbng_status_string": (ctypes.c_char_p, [_I32]),
    "pbng_last_error": (ctypes.c_char_p, [_P]),
    "pbng_destroy": (None, [_P]),
}

_lib = None


def load():
    """Loads libpbng.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with paper_2306_09021_gb300.build.build() "
            "(there is no non-CUDA implementation)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status, where, handle=None):
    if status != PBNG_OK:
        detail = ""
        if handle:
            detail = (load().pbng_last_error(handle) or b"").decode(errors="replace")
        raise PbngError(status, where, detail)
