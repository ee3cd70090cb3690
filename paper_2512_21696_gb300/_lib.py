"""ctypes view of the C ABI declared in include/lbm.h (structures + symbols).

Only argument marshalling lives here; every step of the method runs in the
CUDA library.  Importing this module does not need a GPU; calling anything
that touches device memory does.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_OOM = -3
LBM_ERR_NUMERIC = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_STATE = -6

LBM_MEM_HOST = 0
LBM_MEM_DEVICE = 1

LBM_CELL_PORE, LBM_CELL_SOLID, LBM_CELL_GRAY, LBM_CELL_INLET, LBM_CELL_OUTLET = 0, 1, 2, 3, 4
LBM_LATTICE_D3Q19, LBM_LATTICE_D2Q9 = 0, 1
LBM_STORAGE_F32, LBM_STORAGE_F16S, LBM_STORAGE_BF16S = 0, 1, 2
LBM_MAX_PORE_TYPES = 16


class lbm_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("periodic", C.c_int * 3),
        ("tau", C.c_double * 2),
        ("G", C.c_double),
        ("kappa_csf", C.c_double),
        ("phi_avg", C.c_double * 2),
        ("phi_max", C.c_double * 2),
        ("csf_everywhere", C.c_int),
        ("rho_wall", C.c_double * 2),
        ("body_accel", (C.c_double * 3) * 2),
        ("wet_idx", C.c_int),
        ("rho_hi", C.c_double), ("rho_lo", C.c_double),
        ("s_lo", C.c_double), ("s_hi", C.c_double),
        ("at_cut", C.c_double),
        ("eps_n", C.c_double),
        ("kr_min", C.c_double),
        ("c_g", C.c_double),
        ("storage", C.c_int),
        ("stream", C.c_void_p),
        ("probe_center", C.c_double * 3),
        ("probe_r_in", C.c_double),
        ("probe_r_out", C.c_double),
        ("lattice", C.c_int),
    ]


class lbm_constitutive(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("kc_d", "pd", "lambda_", "swr", "nw", "nn", "phi_ref",
                                          "pc_ref_max_f", "pc_ref_min_f", "aniso", "thomeer_g")]


class lbm_obs(C.Structure):
    _fields_ = [
        ("mass", C.c_double * 2),
        ("sat", C.c_double),
        ("flux_out", C.c_double),
        ("flux_vol", C.c_double * 3),
        ("max_u", C.c_double),
        ("dp", C.c_double),
        ("nan_count", C.c_longlong),
        ("step", C.c_longlong),
    ]


class lbm_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("total_ms", C.c_double)]


class lbm_loss(C.Structure):
    _fields_ = [("q_target", C.c_double), ("s_target", C.c_double)]


EXPORTS = [
    "lbm_strerror", "lbm_last_cuda_error", "lbm_abi_version", "lbm_default_params",
    "lbm_default_constitutive", "lbm_create", "lbm_destroy", "lbm_set_constitutive",
    "lbm_set_geometry", "lbm_init_fields", "lbm_step", "lbm_observables", "lbm_get_fields",
    "lbm_get_static", "lbm_state_size", "lbm_save_state", "lbm_load_state", "lbm_profile",
    "lbm_profile_read", "lbm_launch_count", "lbm_struct_size", "lbm_observables_noalloc", "lbm_set_kernel",
    "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_run", "lbm_batch_step", "lbm_batch_tune", "lbm_batch_info",
    "lbm_adjoint_run", "lbm_batch_observables", "lbm_batch_step_to_steady", "lbm_set_pressure",
    "lbm_pressure_levels", "lbm_set_mss", "lbm_mss_to_saturation", "lbm_batch_mss_to_saturation",
    "lbm_observables_async", "lbm_obs_decode", "lbm_inject_launch_failures", "lbm_get_kernel",
]
LBM_OBS_RAW = 17

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_needed: bool = True):
    """Load liblbm.so (building it with nvcc first if missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is not built; run paper_2512_21696_gb300.build.build()")
        lib = C.CDLL(path)
        P = C.c_void_p
        vp = C.c_void_p
        lib.lbm_strerror.restype = C.c_char_p
        lib.lbm_strerror.argtypes = [C.c_int]
        lib.lbm_last_cuda_error.restype = C.c_char_p
        lib.lbm_last_cuda_error.argtypes = []
        lib.lbm_abi_version.restype = C.c_int
        lib.lbm_default_params.argtypes = [C.POINTER(lbm_params), C.c_int, C.c_int, C.c_int]
        lib.lbm_default_constitutive.argtypes = [C.POINTER(lbm_constitutive)]
        lib.lbm_create.argtypes = [C.POINTER(P), C.POINTER(lbm_params)]
        lib.lbm_destroy.argtypes = [P]
        lib.lbm_set_constitutive.argtypes = [P, C.c_int, C.POINTER(lbm_constitutive)]
        lib.lbm_set_geometry.argtypes = [P, vp, vp, vp, C.c_int]
        lib.lbm_init_fields.argtypes = [P, vp, vp, vp, C.c_int]
        lib.lbm_step.argtypes = [P, C.c_int]
        lib.lbm_observables.argtypes = [P, C.POINTER(lbm_obs)]
        lib.lbm_get_fields.argtypes = [P, vp, vp, vp, vp, C.c_int]
        lib.lbm_get_static.argtypes = [P, vp, vp, vp, vp, C.c_int]
        lib.lbm_state_size.argtypes = [P, C.POINTER(C.c_size_t)]
        lib.lbm_save_state.argtypes = [P, vp, C.c_size_t]
        lib.lbm_load_state.argtypes = [P, vp, C.c_size_t]
        lib.lbm_profile.argtypes = [P, C.c_int]
        lib.lbm_profile_read.argtypes = [P, C.POINTER(lbm_kernel_stat), C.c_int, C.POINTER(C.c_int)]
        lib.lbm_launch_count.argtypes = [P, C.POINTER(C.c_longlong)]
        lib.lbm_observables_noalloc.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_double,
                                                C.POINTER(C.c_double), vp, C.POINTER(lbm_obs)]
        lib.lbm_set_kernel.argtypes = [P, C.c_int, C.c_int]
        lib.lbm_get_kernel.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.lbm_inject_launch_failures.argtypes = [P, C.c_int]
        lib.lbm_set_pressure.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.lbm_set_mss.argtypes = [P, C.c_double]
        lib.lbm_observables_async.argtypes = [P, C.c_void_p]
        lib.lbm_obs_decode.argtypes = [P, C.c_void_p, C.c_void_p]
        lib.lbm_mss_to_saturation.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                              C.POINTER(C.c_int)]
        lib.lbm_batch_mss_to_saturation.argtypes = [P, C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double,
                                                    C.c_int, C.c_int, C.POINTER(C.c_int)]
        lib.lbm_pressure_levels.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                                            C.c_double, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        lib.lbm_adjoint_run.argtypes = [P, C.POINTER(lbm_loss), C.c_int, C.c_int, vp, C.c_int,
                                        C.POINTER(C.c_double)]
        lib.lbm_batch_observables.argtypes = [P, C.POINTER(lbm_obs)]
        lib.lbm_batch_step_to_steady.argtypes = [P, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int)]
        lib.lbm_batch_create.argtypes = [C.POINTER(P), C.c_int, C.POINTER(lbm_params)]
        lib.lbm_batch_destroy.argtypes = [P]
        lib.lbm_batch_run.argtypes = [P, C.c_int, C.POINTER(P)]
        lib.lbm_batch_step.argtypes = [P, C.c_int]
        lib.lbm_batch_tune.argtypes = [P, C.c_int, C.POINTER(C.c_int)]
        lib.lbm_batch_info.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_longlong), C.POINTER(C.c_int)]
        lib.lbm_struct_size.restype = C.c_size_t
        lib.lbm_struct_size.argtypes = [C.c_int]
        for name in EXPORTS:
            if name not in ("lbm_strerror", "lbm_last_cuda_error", "lbm_struct_size"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib
