"""ctypes declarations of the C ABI in include/fullwave_gb.h (argument
marshalling only; every computation runs inside libfullwave_gb.so)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfullwave_gb.so")
MAX_MECH = 4
MAX_W = 8

FW_OK = 0
FW_ERR_ARG = -1
FW_ERR_CUDA = -2
FW_ERR_NOMEM = -3
FW_ERR_UNSTABLE = -4
FW_ERR_STATE = -5
FW_ERR_UNSUPPORTED = -6
FW_ERR_SIZE = -7
FW_CANCELLED = -8
FW_SERVER_MAX_SKIPS = 8
FW_NOALLOC_MAX_BYTES = 64 << 20

FW_STORE_F32, FW_STORE_BF16, FW_STORE_F16, FW_STORE_F64 = 0, 1, 2, 3
FW_FIELD_P, FW_FIELD_V, FW_FIELD_PSI1, FW_FIELD_PSI2, FW_FIELD_PSI1P, FW_FIELD_PSI2P = range(6)


class fw_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dt", C.c_double), ("cfl", C.c_double),
                ("pml", C.c_int), ("transition", C.c_int), ("f0", C.c_double), ("pml_r0", C.c_double),
                ("layer_relax", C.c_int), ("time_order", C.c_int)]


class fw_relax_params(C.Structure):
    _fields_ = [("n_mech", C.c_int), ("kappa1", C.c_double), ("kappa2", C.c_double),
                ("d1", C.c_double * MAX_MECH), ("alpha1", C.c_double * MAX_MECH),
                ("d2", C.c_double * MAX_MECH), ("alpha2", C.c_double * MAX_MECH)]


class fw_fit_opts(C.Structure):
    _fields_ = [("f_min", C.c_double), ("f_max", C.c_double), ("n_freq", C.c_int), ("n_w", C.c_int),
                ("w", C.c_double * MAX_W), ("maxiter", C.c_int), ("xatol", C.c_double),
                ("fatol", C.c_double), ("f_ref", C.c_double), ("c0", C.c_double), ("n_threads", C.c_int)]


class fw_fit_report(C.Structure):
    _fields_ = [("J", C.c_double), ("w", C.c_double), ("nrmse", C.c_double), ("disp_rmse", C.c_double),
                ("failed", C.c_int), ("n_iter", C.c_int), ("n_eval", C.c_int)]


class fw_medium_info(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("n_mech", C.c_int),
                ("storage", C.c_int), ("n_classes", C.c_int), ("nonlinear", C.c_int),
                ("dx", C.c_double), ("dt", C.c_double), ("c_max", C.c_double), ("ceff_max", C.c_double),
                ("device_bytes", C.c_size_t), ("step", C.c_longlong),
                ("n_src", C.c_int), ("n_rcv", C.c_int), ("n_rec", C.c_int), ("time_order", C.c_int)]


class fw_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("chunk_steps", C.c_int),
                ("n_streams", C.c_int), ("policy", C.c_int), ("short_work", C.c_double)]


class fw_request(C.Structure):
    _fields_ = [("grid", fw_grid), ("c", C.c_void_p), ("rho", C.c_void_p), ("beta", C.c_void_p),
                ("class_idx", C.c_void_p), ("classes", C.POINTER(fw_relax_params)), ("n_classes", C.c_int),
                ("storage", C.c_int), ("src_mask", C.c_void_p), ("waveforms", C.c_void_p), ("n_wave", C.c_int),
                ("wave_of", C.c_void_p), ("rcv_mask", C.c_void_p), ("decim", C.c_int), ("n_steps", C.c_int),
                ("traces_out", C.c_void_p), ("tag", C.c_longlong)]


class fw_completion(C.Structure):
    _fields_ = [("id", C.c_longlong), ("tag", C.c_longlong), ("status", C.c_int), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("voxel_steps", C.c_longlong),
                ("max_abs_p", C.c_float)]


class fw_server_stats(C.Structure):
    _fields_ = [("queued", C.c_int), ("building", C.c_int), ("active", C.c_int), ("done", C.c_int),
                ("bytes_reserved", C.c_size_t), ("bytes_budget", C.c_size_t), ("bytes_largest_free", C.c_size_t)]


OBJFN = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_double), C.c_void_p)
ALLOCFN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREEFN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.c_int

# name -> (restype, argtypes); every symbol declared in include/fullwave_gb.h
SIGNATURES = {
    "fw_fit_default_opts": (None, [C.POINTER(fw_fit_opts)]),
    "fw_fit_relaxation": (_I, [C.c_double, C.c_double, _I, C.POINTER(fw_fit_opts),
                               C.POINTER(fw_relax_params), C.POINTER(fw_fit_report)]),
    "fw_fit_objective": (_I, [C.c_double, C.c_double, C.c_double, C.POINTER(fw_fit_opts), _D, _I, _D]),
    "fw_fit_targets": (_I, [C.c_double, C.c_double, C.c_double, C.c_double, _D, _I, _D, _D]),
    "fw_model_wavenumber": (_I, [C.POINTER(fw_relax_params), C.c_double, _D, _I, _D, _D]),
    "fw_nelder_mead": (_I, [_I, _D, _D, _D, OBJFN, _P, _I, C.c_double, C.c_double, _D,
                            C.POINTER(_I), C.POINTER(_I)]),
    "fw_set_allocator": (None, [ALLOCFN, FREEFN, _P]),
    "fw_medium_bytes": (_I, [C.POINTER(fw_grid), _I, _I, _I, C.POINTER(C.c_size_t)]),
    "fw_create_medium": (_I, [C.POINTER(fw_grid), _P, _P, _P, _P, _P, _I, _I, C.POINTER(fw_fit_opts), _P,
                              C.POINTER(_P)]),
    "fw_create_medium_classes": (_I, [C.POINTER(fw_grid), _P, _P, _P, _P, C.POINTER(fw_relax_params), _I, _I,
                                      _P, C.POINTER(_P)]),
    "fw_set_sources": (_I, [_P, _P, _P, _I, _I, _P]),
    "fw_set_receivers": (_I, [_P, _P, _I, _I]),
    "fw_step": (_I, [_P, _I, _P]),
    "fw_run": (_I, [_P, _I, _P]),
    "fw_step_timed": (_I, [_P, _I, _P, _D, _D, _D, _D, C.POINTER(_I)]),
    "fw_set_waveform_samples": (_I, [_P, _I, _I, _P, _P]),
    "fw_read_receivers_range": (_I, [_P, _I, _I, _P, _P]),
    "fw_read_field": (_I, [_P, _I, _I, _P, _I, _P]),
    "fw_read_field_noalloc": (_I, [_P, _I, _I, _P, _I, _P]),
    "fw_write_field": (_I, [_P, _I, _I, _P, _I, _P]),
    "fw_read_receivers": (_I, [_P, _P, _I, _P]),
    "fw_state_bytes": (_I, [_P, C.POINTER(C.c_size_t)]),
    "fw_save_state": (_I, [_P, _P, _P]),
    "fw_load_state": (_I, [_P, _P, _P]),
    "fw_gradient": (_I, [_P, _I, _I, _P, _P, _P, _P, _I, _P]),
    "fw_status": (_I, [_P, C.POINTER(C.c_float)]),
    "fw_medium_get_info": (_I, [_P, C.POINTER(fw_medium_info)]),
    "fw_destroy_medium": (None, [_P]),
    "fw_server_create": (_I, [C.POINTER(fw_server_opts), C.POINTER(_P)]),
    "fw_server_submit": (_I, [_P, C.POINTER(fw_request), C.POINTER(C.c_longlong)]),
    "fw_server_poll": (_I, [_P, C.POINTER(fw_completion), _I, C.POINTER(_I), C.c_double]),
    "fw_server_cancel": (_I, [_P, C.c_longlong]),
    "fw_server_stats_get": (_I, [_P, C.POINTER(fw_server_stats)]),
    "fw_server_now": (C.c_double, [_P]),
    "fw_server_destroy": (None, [_P]),
    "fw_strerror": (C.c_char_p, [_I]),
    "fw_version": (_I, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfullwave_gb.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libfullwave_gb.so is not built (run paper_2606_11103_gb300.build.build() "
                           "or __graft_entry__.build()); there is no fallback path")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FwError(RuntimeError):
    def __init__(self, code, what=""):
        msg = load().fw_strerror(code).decode()
        super().__init__("%s: %s (%d)" % (what, msg, code) if what else "%s (%d)" % (msg, code))
        self.code = code


def check(code, what=""):
    if code != FW_OK:
        raise FwError(code, what)
    return code
