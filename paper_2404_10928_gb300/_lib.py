"""ctypes binding of the C ABI in ``include/pa.h`` (argument marshalling only).

The names, argument order and structures mirror the header one to one.  The
shared library is ``libpa.so`` next to this file, built by ``build.py``; there
is no fallback: if it is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# PA_LIB_PATH selects another build of the same library (the index-checked
# libpa_checked.so, say); it must export the same entry points
LIB_PATH = os.environ.get("PA_LIB_PATH") or os.path.join(HERE, "libpa.so")

c_int, c_double, c_void_p, c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64

PA_OK = 0
PA_ERR_INVALID_ARG = 1
PA_ERR_GEOMETRY = 2
PA_ERR_CUDA = 3
PA_ERR_OOM = 4
PA_ERR_TIMEOUT = 5
PA_ERR_DEVICE_CHECK = 6
PA_ERR_UNSUPPORTED = 7

PA_LANDWEBER = 0
PA_CGLS = 1
PA_FISTA = 2
PA_PCGLS = 3
PA_BP_NONE = 0
PA_BP_UBP = 1
PA_F32 = 0
PA_F16 = 1
PA_F64 = 2


class pa_grid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int),
                ("dx", c_double), ("dy", c_double), ("dz", c_double),
                ("origin", c_double * 3)]


class pa_plan_opts(ctypes.Structure):
    _fields_ = [("t0", c_double), ("amp_scale", c_double), ("y_dtype", c_int),
                ("adj_cluster", c_int), ("fwd_sensors_per_cta", c_int), ("fwd_threads", c_int),
                ("adj_warps", c_int)]


class pa_recon_opts(ctypes.Structure):
    _fields_ = [("omega", c_double), ("nonneg", c_int), ("power_iters", c_int),
                ("power_v0_dev", c_void_p), ("residual_history_host", ctypes.POINTER(c_double)),
                ("use_graph", c_int), ("kernel_timing", c_int), ("l1_weight", c_double),
                ("tv_weight", c_double), ("tv_eps", c_double), ("restart", c_int)]


class pa_plan_info(ctypes.Structure):
    _fields_ = [("n_pixels", c_int64), ("n_sensors", c_int64), ("n_samples", c_int64),
                ("pairs", c_int64), ("tile", c_int * 3), ("window", c_int), ("cluster", c_int),
                ("fwd_sensors", c_int), ("device_bytes", c_int64), ("fwd_threads", c_int),
                ("adj_warps", c_int)]


_P = c_void_p  # opaque pa_plan*
_STREAM = c_void_p
_DP = ctypes.POINTER(c_double)

# name -> (restype, argtypes), exactly the declarations of include/pa.h
SIGNATURES = {
    "pa_recon_opts_default": (None, [ctypes.POINTER(pa_recon_opts)]),
    "pa_plan_create": (c_int, [ctypes.POINTER(_P), _DP, c_int, ctypes.POINTER(pa_grid), c_double,
                               c_double, c_int, ctypes.POINTER(pa_plan_opts)]),
    "pa_plan_destroy": (c_int, [_P]),
    "pa_plan_set_sound_speed": (c_int, [_P, c_double]),
    "pa_plan_sync_status": (c_int, [_P]),
    "pa_plan_query": (c_int, [_P, ctypes.POINTER(pa_plan_info)]),
    "pa_forward": (c_int, [_P, c_void_p, c_void_p, _STREAM]),
    "pa_adjoint": (c_int, [_P, c_void_p, c_void_p, _STREAM]),
    "pa_backproject": (c_int, [_P, c_void_p, c_int, c_void_p, _STREAM]),
    "pa_dense_assemble": (c_int, [_P, c_int, c_void_p, _STREAM]),
    "pa_freq_forward": (c_int, [_P, c_int, c_double, c_double, c_void_p, c_void_p, _STREAM]),
    "pa_freq_adjoint": (c_int, [_P, c_int, c_double, c_double, c_void_p, c_void_p, _STREAM]),
    "pa_dense_matvec": (c_int, [_P, c_int, c_void_p, c_int, c_void_p, c_void_p, _STREAM]),
    "pa_power_iteration": (c_int, [_P, c_int, c_void_p, _DP, _STREAM]),
    "pa_reconstruct": (c_int, [_P, c_int, c_int, c_void_p, c_void_p,
                               ctypes.POINTER(pa_recon_opts), _STREAM]),
    "pa_reconstruct_host": (c_int, [_P, c_int, c_int, c_void_p, c_void_p,
                                    ctypes.POINTER(pa_recon_opts), _STREAM]),
    "pa_plan_kernel_times": (c_int, [_P, _DP, ctypes.POINTER(c_int), _DP, ctypes.POINTER(c_int)]),
    "pa_plan_time_gathers": (c_int, [_P, c_int, c_void_p, c_void_p, _DP, _DP, _STREAM]),
    "pa_shard_cgls_begin": (c_int, [_P, c_int, c_void_p, c_void_p, c_void_p, c_int, _STREAM]),
    "pa_shard_cgls_direction": (c_int, [_P, c_int, c_void_p, c_void_p, c_int, _STREAM]),
    "pa_shard_cgls_update": (c_int, [_P, c_int, c_void_p, c_void_p, c_void_p, c_int, _STREAM]),
    "pa_shard_cgls_finish": (c_int, [_P, c_void_p, c_int, c_void_p, c_int, _STREAM]),
    "pa_dc": (c_int, [_P, c_void_p, c_void_p, c_void_p, _STREAM]),
    "pa_batch_create": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int]),
    "pa_batch_destroy": (c_int, [c_void_p]),
    "pa_batch_landweber": (c_int, [c_void_p, c_int, ctypes.POINTER(c_void_p),
                                   ctypes.POINTER(c_void_p), _DP, c_int, _DP, _STREAM]),
    "pa_batch_set_wait_limit": (c_int, [c_void_p, c_double]),
    "pa_batch_reconstruct": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(c_void_p),
                                     ctypes.POINTER(c_void_p), _DP, c_int, _DP, _STREAM]),
    "pa_debug_fail_allocations": (c_int, [ctypes.c_longlong]),
    "pa_tv": (c_int, [_P, c_void_p, c_double, c_void_p, c_void_p, _STREAM]),
    "pa_forward_frames": (c_int, [_P, c_int, c_void_p, c_void_p, _STREAM]),
    "pa_adjoint_frames": (c_int, [_P, c_int, c_void_p, c_void_p, _STREAM]),
    "pa_residual_frames": (c_int, [_P, c_int, c_void_p, c_void_p, c_void_p, c_void_p, _STREAM]),
    "pa_adjoint_axpy_frames": (c_int, [_P, c_int, c_void_p, c_void_p, c_double, c_void_p,
                                       c_double, c_int, c_void_p, _STREAM]),
    "pa_dc_frames": (c_int, [_P, c_int, c_void_p, c_void_p, c_double, c_int, c_void_p, _STREAM]),
    "pa_tv_frames": (c_int, [_P, c_int, c_void_p, c_double, c_void_p, c_void_p, _STREAM]),
    "pa_landweber_step_frames": (c_int, [_P, c_int, c_void_p, c_void_p, c_double, c_int,
                                         c_void_p, _STREAM]),
    "pa_landweber_step_vjp_frames": (c_int, [_P, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                             c_double, c_int, c_void_p, c_void_p, c_void_p,
                                             _STREAM]),
    "pa_data_tv_loss_frames": (c_int, [_P, c_int, c_void_p, c_void_p, c_double, c_double,
                                       c_void_p, c_void_p, c_void_p, _STREAM]),
    "pa_data_tv_loss_vjp_frames": (c_int, [_P, c_int, c_void_p, c_void_p, c_void_p, c_double,
                                           c_double, c_void_p, c_void_p, _STREAM]),
    "pa_adjoint_static": (c_int, [_DP, c_int, ctypes.POINTER(pa_grid), c_double, c_double, c_int,
                                  ctypes.POINTER(pa_plan_opts), c_void_p, c_void_p, _STREAM]),
    "pa_status_string": (ctypes.c_char_p, [c_int]),
    "pa_last_error": (ctypes.c_char_p, []),
    "pa_version": (c_int, []),
}

_lib = None


class PAError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {message} (status {status})")


def load():
    """Load libpa.so (raises if it is not built; there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2404_10928_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, where: str):
    if status != PA_OK:
        lib = load()
        msg = lib.pa_last_error().decode(errors="replace")
        raise PAError(status, where, msg or lib.pa_status_string(status).decode())
