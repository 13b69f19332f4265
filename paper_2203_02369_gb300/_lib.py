"""ctypes binding of libhamlet (include/hamlet.h): argument marshalling only.

Every computation runs in the CUDA library; if the library is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as ct
import os

from . import build as _build

c_double_p = ct.POINTER(ct.c_double)


class hm_problem_desc(ct.Structure):
    _fields_ = [
        ("N", ct.c_int32), ("precision", ct.c_int32),
        ("L", ct.c_double), ("observer", ct.c_double * 3),
        ("observer_set", ct.c_int32), ("prior_kind", ct.c_int32),
        ("omega_m", ct.c_double), ("omega_b", ct.c_double), ("h", ct.c_double),
        ("n_s", ct.c_double), ("sigma8", ct.c_double), ("T_cmb", ct.c_double),
        ("f_growth", ct.c_double), ("sigma_nl", ct.c_double),
        ("prior_d0", ct.c_double), ("prior_bin", ct.c_double),
        ("prior_nbins", ct.c_int32), ("pad0", ct.c_int32),
        ("prior_logdens_host", c_double_p),
        ("prior_alpha", ct.c_double), ("prior_dmin", ct.c_double), ("prior_dmax", ct.c_double),
        ("device", ct.c_int32), ("pad1", ct.c_int32),
        ("prior_pad", ct.c_double),
    ]


class hm_problem_info(ct.Structure):
    _fields_ = [
        ("N", ct.c_int32), ("precision", ct.c_int32), ("n_points", ct.c_int64),
        ("L", ct.c_double), ("delta", ct.c_double), ("f_growth", ct.c_double),
        ("sigma_v", ct.c_double), ("minv_d", ct.c_double), ("pk_amplitude", ct.c_double),
        ("grid_bytes", ct.c_int64), ("spectrum_bytes", ct.c_int64),
    ]


class hm_trace(ct.Structure):
    _fields_ = [
        ("traj", ct.c_int64), ("H_old", ct.c_double), ("H_new", ct.c_double),
        ("logu", ct.c_double), ("psi", ct.c_double), ("eps", ct.c_double), ("accept", ct.c_int32),
        ("status", ct.c_int32),
    ]


HM_OK, HM_EINVAL, HM_ENOMEM, HM_ECUDA, HM_EDOMAIN, HM_ESTATE = 0, -1, -2, -3, -4, -5
HM_FP32, HM_FP64 = 0, 1
HM_PRIOR_TABLE, HM_PRIOR_POWER, HM_PRIOR_DZ = 0, 1, 2

# (name, restype, argtypes) of every exported entry point
_P = ct.c_void_p
SIGNATURES = [
    ("hm_supported", ct.c_int, [ct.c_int32, ct.c_int32]),
    ("hm_init_problem", ct.c_int, [ct.POINTER(hm_problem_desc), ct.POINTER(_P)]),
    ("hm_destroy_problem", None, [_P]),
    ("hm_problem_get_info", ct.c_int, [_P, ct.POINTER(hm_problem_info)]),
    ("hm_set_catalog", ct.c_int, [_P, ct.c_int64, c_double_p, c_double_p, c_double_p, c_double_p, c_double_p]),
    ("hm_set_catalog_sg", ct.c_int, [_P, ct.c_int64, c_double_p, c_double_p, c_double_p, c_double_p, c_double_p,
                                     c_double_p]),
    ("hm_logpost_grad", ct.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("hm_logpost_grad_noalloc", ct.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("hm_problem_last_status", ct.c_int, [_P, _P, ct.POINTER(ct.c_int32)]),
    ("hm_device_wait_timeouts", ct.c_int, [ct.c_int32, ct.c_int32, ct.POINTER(ct.c_int32)]),
    ("hm_problem_prior_table", ct.c_int, [_P, ct.c_int32, c_double_p, ct.POINTER(ct.c_int32), c_double_p,
                                          c_double_p]),
    ("hm_velocity_field", ct.c_int, [_P, _P, _P, _P]),
    ("hm_fft_r2c", ct.c_int, [_P, _P, _P, ct.c_int32, _P]),
    ("hm_fft_c2r", ct.c_int, [_P, _P, _P, ct.c_int32, _P]),
    ("hm_cells", ct.c_int, [_P, _P, _P, _P, _P]),
    ("hm_state_create", ct.c_int, [_P, ct.c_uint64, c_double_p, ct.POINTER(_P)]),
    ("hm_state_create_batch", ct.c_int, [ct.POINTER(_P), ct.c_int32, ct.c_int32, ct.POINTER(ct.c_int32),
                                         ct.POINTER(ct.c_int32), ct.c_uint64, ct.POINTER(c_double_p),
                                         ct.POINTER(_P)]),
    ("hm_destroy_state", None, [_P]),
    ("hm_state_set", ct.c_int, [_P, ct.c_int32, _P, _P, _P, _P, _P]),
    ("hm_state_get", ct.c_int, [_P, ct.c_int32, _P, _P, _P, _P, _P]),
    ("hm_state_get_grad", ct.c_int, [_P, ct.c_int32, _P, _P, _P]),
    ("hm_state_refresh", ct.c_int, [_P, _P]),
    ("hm_state_scalars", ct.c_int, [_P, ct.c_int32, c_double_p, c_double_p, ct.POINTER(ct.c_int64), _P]),
    ("hm_state_set_traj", ct.c_int, [_P, ct.c_int32, ct.c_int64]),
    ("hm_leapfrog", ct.c_int, [_P, ct.c_int32, ct.c_double, ct.c_int32, _P]),
    ("hm_run_chain", ct.c_int, [_P, ct.c_int32, ct.c_int32, c_double_p, ct.c_int32, ct.c_int32,
                                ct.POINTER(hm_trace), _P]),
    ("hm_slots_create", ct.c_int, [_P, ct.c_int32, ct.c_int64, ct.c_uint64, ct.POINTER(_P)]),
    ("hm_slots_count", ct.c_int, [_P, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32)]),
    ("hm_slots_load", ct.c_int, [_P, _P, ct.c_int32, c_double_p, ct.c_double, ct.c_double, ct.c_double,
                                 ct.POINTER(ct.c_int32), _P]),
    ("hm_slots_adapt_end", ct.c_int, [_P, ct.c_int32, c_double_p, _P]),
    ("hm_slots_release", ct.c_int, [_P, ct.c_int32, ct.POINTER(ct.c_int32), _P]),
    ("hm_slots_run", ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_int32, ct.POINTER(hm_trace), _P]),
    ("hm_state_sample_sigma_nl", ct.c_int, [_P, ct.c_int32, c_double_p, _P]),
    ("hm_state_get_sigma_nl", ct.c_int, [_P, c_double_p, c_double_p, _P]),
    ("hm_adapt_step_size", ct.c_int, [_P, ct.c_int32, ct.c_int32, ct.c_double, c_double_p, ct.c_int32,
                                      c_double_p, ct.POINTER(hm_trace), _P]),
    ("hm_state_analytics", ct.c_int, [_P, ct.c_int32, ct.c_int32, c_double_p, ct.c_int32, _P]),
    ("hm_state_analytics_read", ct.c_int, [_P, ct.c_int32, _P, _P, _P, _P, c_double_p, ct.c_int32, c_double_p,
                                           ct.POINTER(ct.c_int64), _P]),
    ("hm_state_profile", ct.c_int, [_P, ct.c_int32]),
    ("hm_state_profile_collect", ct.c_int, [_P]),
    ("hm_state_profile_read", ct.c_int, [_P, ct.c_int32, c_double_p, ct.POINTER(ct.c_int64),
                                         ct.POINTER(ct.c_int32)]),
    ("hm_kernel_kind_name", ct.c_char_p, [ct.c_int32]),
    ("hm_dz_prior_table", ct.c_int, [ct.c_double, ct.c_int64, c_double_p, ct.c_double, ct.c_double, ct.c_int32,
                                     c_double_p, ct.POINTER(ct.c_int32)]),
    ("hm_philox", ct.c_int, [ct.c_uint64, ct.c_int64, ct.c_uint32, ct.c_uint32, ct.c_uint32, _P, _P]),
    ("hm_last_error", ct.c_char_p, []),
]


class HamletError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libhamlet error {code}: {msg}")
        self.code = code


_LIB = None


def library_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhamlet.so (building it in-tree first if it is absent)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build_library()
    if not os.path.exists(path):
        raise HamletError(HM_ESTATE, f"libhamlet.so not found at {path}; run build_library()")
    lib = ct.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def check(rc):
    if rc != HM_OK:
        raise HamletError(rc, _LIB.hm_last_error().decode(errors="replace"))
    return rc
