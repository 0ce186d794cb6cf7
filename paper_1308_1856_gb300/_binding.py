"""ctypes binding of libtdse (include/tdse.h), argument marshalling only.

The functions carry the C names and signatures.  Every step of the
propagation runs in the CUDA library; this module only converts arguments.
Importing it fails loudly when the shared library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

TDSE_OK = 0
TDSE_ERR_ARG = -1
TDSE_ERR_OOM = -2
TDSE_ERR_CUDA = -3
TDSE_ERR_NONFINITE = -4
TDSE_ERR_STATE = -7
TDSE_STENCIL_3, TDSE_STENCIL_5 = 3, 5
TDSE_TAYLOR, TDSE_RK4, TDSE_LANCZOS = 0, 1, 2
TDSE_GHOST_ZERO, TDSE_GHOST_ODD = 0, 1
TDSE_FP64, TDSE_MIXED = 0, 1
(TDSE_RK_EULER, TDSE_RK_CLASSIC, TDSE_RK_FEHLBERG, TDSE_RK_CASH_KARP, TDSE_RK_DORMAND_PRINCE,
 TDSE_RK_MERSON) = range(6)
TDSE_GAUGE_LENGTH, TDSE_GAUGE_VELOCITY = 0, 1
TDSE_PULSE_SIN2_E, TDSE_PULSE_SIN2_A = 0, 1
TDSE_MAX_KRYLOV = 32
TDSE_SMALL_GRID_AUTO, TDSE_SMALL_GRID_OFF, TDSE_SMALL_GRID_FORCE = 0, 1, 2

# Every symbol include/tdse.h declares: name -> (restype, argtypes)
_c_int, _c_double, _c_long, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


class tdse_opts(ctypes.Structure):
    _fields_ = [("ghost", ctypes.c_int), ("offset", ctypes.c_double), ("absorber", ctypes.c_int),
                ("absorber_r", ctypes.c_double), ("r_b", ctypes.c_double),
                ("precision", ctypes.c_int), ("gauge", ctypes.c_int)]


class tdse_instance_spec(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("dr", ctypes.c_double), ("lmax", ctypes.c_int),
                ("Z", ctypes.c_double), ("E0", ctypes.c_double), ("omega", ctypes.c_double),
                ("ncycles", ctypes.c_double), ("cep", ctypes.c_double), ("krylov", ctypes.c_int),
                ("dt", ctypes.c_double), ("absorber_r", ctypes.c_double), ("r_b", ctypes.c_double),
                ("gauge", ctypes.c_int), ("pulse_shape", ctypes.c_int)]


class tdse_schedule(ctypes.Structure):
    _fields_ = [("prefetch_rows", ctypes.c_int), ("ring_rows", ctypes.c_int),
                ("stencil_blocks_per_sm", ctypes.c_int), ("elem_blocks_per_sm", ctypes.c_int)]


class tdse_server_stats_t(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_longlong), ("running", ctypes.c_longlong),
                ("resident", ctypes.c_longlong), ("finished_total", ctypes.c_longlong),
                ("bytes_budget", ctypes.c_ulonglong), ("bytes_in_use", ctypes.c_ulonglong),
                ("largest_free", ctypes.c_ulonglong), ("gp_steps", ctypes.c_longlong),
                ("launches", ctypes.c_longlong)]


_llp = ctypes.POINTER(ctypes.c_longlong)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)

SIGNATURES = {
    "tdse_create": (_c_int, [_c_int, _c_double, _c_int, _c_int, _c_double, _dp,
                             ctypes.POINTER(_vp)]),
    "tdse_destroy": (_c_int, [_vp]),
    "tdse_last_error": (ctypes.c_char_p, [_vp]),
    "tdse_set_options": (_c_int, [_vp, ctypes.POINTER(tdse_opts)]),
    "tdse_set_stream": (_c_int, [_vp, _vp]),
    "tdse_set_pulse": (_c_int, [_vp, _c_double, _c_double, _c_double, _c_double]),
    "tdse_field": (_c_double, [_vp, _c_double]),
    "tdse_vector_potential": (_c_double, [_vp, _c_double]),
    "tdse_set_pulse_shape": (_c_int, [_vp, _c_int]),
    "tdse_set_time": (_c_int, [_vp, _c_double]),
    "tdse_get_time": (_c_double, [_vp]),
    "tdse_set_state": (_c_int, [_vp, _vp]),
    "tdse_get_state": (_c_int, [_vp, _vp]),
    "tdse_set_state_device": (_c_int, [_vp, _vp]),
    "tdse_get_state_device": (_c_int, [_vp, _vp]),
    "tdse_set_reference": (_c_int, [_vp, _vp]),
    "tdse_propagate": (_c_int, [_vp, _c_int, _c_int, _c_double, _c_long]),
    "tdse_propagate_imag": (_c_int, [_vp, _c_int, _c_int, _c_double, _c_long, _dp]),
    "tdse_propagate_rk": (_c_int, [_vp, _c_int, _c_double, _c_long, _dp]),
    "tdse_dipole_moments": (_c_int, [_vp, _dp, _dp, _dp]),
    "tdse_dipole_series": (_c_int, [_vp, _c_long]),
    "tdse_dipole_series_read": (_c_int, [_vp, _dp, _c_long, ctypes.POINTER(_c_long)]),
    "tdse_flux_setup": (_c_int, [_vp, _c_double, _c_int, _dp]),
    "tdse_check_guards": (_c_int, [_vp]),
    "tdse_record_setup": (_c_int, [_vp, _c_long, _c_long]),
    "tdse_record_width": (_c_long, [_vp]),
    "tdse_record_read": (_c_int, [_vp, _dp, _c_long, ctypes.POINTER(_c_long)]),
    "tdse_checkpoint_bytes": (ctypes.c_size_t, [_vp]),
    "tdse_checkpoint_save": (_c_int, [_vp, _vp, ctypes.c_size_t]),
    "tdse_checkpoint_load": (_c_int, [_vp, _vp, ctypes.c_size_t]),
    "tdse_flux_read": (_c_int, [_vp, _dp, _dp, _dp, _dp]),
    "tdse_observables": (_c_int, [_vp, _dp, _vp, _dp, _dp, _dp]),
    "tdse_apply_h": (_c_int, [_vp, _c_double, _vp, _vp]),
    "tdse_sync": (_c_int, [_vp]),
    "tdse_fma_throughput": (_c_int, [_c_int, _dp, _vp]),
    "tdse_lanczos_expm": (_c_int, [_c_int, _dp, _dp, _c_double, _c_int, _dp, ctypes.POINTER(_c_int)]),
    "tdse_set_small_grid_path": (_c_int, [_vp, _c_int]),
    "tdse_small_grid_path_used": (_c_int, [_vp]),
    "tdse_set_persistent_path": (_c_int, [_vp, _c_int]),
    "tdse_persistent_path_used": (_c_int, [_vp]),
    "tdse_launch_count": (ctypes.c_longlong, [_vp]),
    "tdse_profile": (_c_int, [_vp, _c_int]),
    "tdse_profile_read": (_c_int, [_vp, _c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "tdse_observables_noalloc": (_c_int, [_c_int, _c_double, _c_int, _c_double, _c_double,
                                          _vp, _vp, _vp, _vp]),
    "tdse_batch_create": (_c_int, [ctypes.POINTER(tdse_instance_spec), _c_int, _c_int, _c_int,
                                   ctypes.POINTER(_vp)]),
    "tdse_batch_destroy": (_c_int, [_vp]),
    "tdse_batch_last_error": (ctypes.c_char_p, [_vp]),
    "tdse_batch_set_stream": (_c_int, [_vp, _vp]),
    "tdse_batch_set_state": (_c_int, [_vp, _c_int, _vp]),
    "tdse_batch_get_state": (_c_int, [_vp, _c_int, _vp]),
    "tdse_batch_get_time": (_c_double, [_vp, _c_int]),
    "tdse_batch_set_time": (_c_int, [_vp, _c_int, _c_double]),
    "tdse_batch_set_states": (_c_int, [_vp, _vp]),
    "tdse_batch_get_states": (_c_int, [_vp, _vp]),
    "tdse_batch_propagate": (_c_int, [_vp, _c_long]),
    "tdse_batch_propagate_io": (_c_int, [_vp, _vp, _vp, _c_long, _c_int]),
    "tdse_batch_observables": (_c_int, [_vp, _c_int, _dp, _vp, _dp, _dp, _dp]),
    "tdse_batch_dipole_series": (_c_int, [_vp, _c_long]),
    "tdse_batch_dipole_series_read": (_c_int, [_vp, _c_int, _dp, _c_long, ctypes.POINTER(_c_long)]),
    "tdse_batch_propagate_imag": (_c_int, [_vp, _c_long, _dp]),
    "tdse_batch_flux_setup": (_c_int, [_vp, _c_int, _dp]),
    "tdse_batch_flux_read": (_c_int, [_vp, _c_int, _dp, _dp, _dp, _dp]),
    "tdse_batch_points": (ctypes.c_longlong, [_vp]),
    "tdse_batch_launch_count": (ctypes.c_longlong, [_vp]),
    "tdse_batch_graph_steps": (ctypes.c_longlong, [_vp]),
    "tdse_batch_profile": (_c_int, [_vp, _c_int]),
    "tdse_batch_profile_read": (_c_int, [_vp, _c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "tdse_batch_autotune": (_c_int, [_vp, ctypes.POINTER(tdse_schedule)]),
    "tdse_batch_set_schedule": (_c_int, [_vp, ctypes.POINTER(tdse_schedule)]),
    "tdse_batch_get_schedule": (_c_int, [_vp, ctypes.POINTER(tdse_schedule)]),
    "tdse_server_autotune": (_c_int, [_vp, ctypes.POINTER(tdse_schedule)]),
    "tdse_server_set_schedule": (_c_int, [_vp, ctypes.POINTER(tdse_schedule)]),
    "tdse_server_instance_bytes": (ctypes.c_ulonglong, [ctypes.POINTER(tdse_instance_spec), _c_int]),
    "tdse_server_create": (_c_int, [ctypes.c_ulonglong, _c_int, _c_int, _c_int, ctypes.POINTER(_vp)]),
    "tdse_server_destroy": (_c_int, [_vp]),
    "tdse_server_last_error": (ctypes.c_char_p, [_vp]),
    "tdse_server_set_stream": (_c_int, [_vp, _vp]),
    "tdse_server_submit": (_c_int, [_vp, ctypes.POINTER(tdse_instance_spec), _c_long, _llp]),
    "tdse_server_step": (_c_int, [_vp, _c_long, _ip]),
    "tdse_server_sync": (_c_int, [_vp]),
    "tdse_server_poll": (_c_int, [_vp, _llp, _c_int, _ip]),
    "tdse_server_status": (_c_int, [_vp, ctypes.c_longlong, _ip, _lp, _lp]),
    "tdse_server_observables": (_c_int, [_vp, ctypes.c_longlong, _dp, _vp, _dp, _dp, _dp]),
    "tdse_server_get_state": (_c_int, [_vp, ctypes.c_longlong, _vp]),
    "tdse_server_release": (_c_int, [_vp, ctypes.c_longlong]),
    "tdse_server_stats": (_c_int, [_vp, ctypes.POINTER(tdse_server_stats_t)]),
    "tdse_server_profile": (_c_int, [_vp, _c_int]),
    "tdse_server_profile_read": (_c_int, [_vp, _c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libtdse.so; raise if it is missing (there is no CPU fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"libtdse is not built ({path}); run paper_1308_1856_gb300/build.py "
                              "or __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _fn(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    return call


tdse_create = _fn("tdse_create")
tdse_destroy = _fn("tdse_destroy")
tdse_last_error = _fn("tdse_last_error")
tdse_set_options = _fn("tdse_set_options")
tdse_set_stream = _fn("tdse_set_stream")
tdse_set_pulse = _fn("tdse_set_pulse")
tdse_field = _fn("tdse_field")
tdse_vector_potential = _fn("tdse_vector_potential")
tdse_set_pulse_shape = _fn("tdse_set_pulse_shape")
tdse_set_time = _fn("tdse_set_time")
tdse_get_time = _fn("tdse_get_time")
tdse_set_state = _fn("tdse_set_state")
tdse_get_state = _fn("tdse_get_state")
tdse_set_state_device = _fn("tdse_set_state_device")
tdse_get_state_device = _fn("tdse_get_state_device")
tdse_set_reference = _fn("tdse_set_reference")
tdse_propagate = _fn("tdse_propagate")
tdse_propagate_imag = _fn("tdse_propagate_imag")
tdse_propagate_rk = _fn("tdse_propagate_rk")
tdse_dipole_moments = _fn("tdse_dipole_moments")
tdse_dipole_series = _fn("tdse_dipole_series")
tdse_dipole_series_read = _fn("tdse_dipole_series_read")
tdse_flux_setup = _fn("tdse_flux_setup")
tdse_check_guards = _fn("tdse_check_guards")
tdse_record_setup = _fn("tdse_record_setup")
tdse_record_width = _fn("tdse_record_width")
tdse_record_read = _fn("tdse_record_read")
tdse_checkpoint_bytes = _fn("tdse_checkpoint_bytes")
tdse_checkpoint_save = _fn("tdse_checkpoint_save")
tdse_checkpoint_load = _fn("tdse_checkpoint_load")
tdse_flux_read = _fn("tdse_flux_read")
tdse_observables = _fn("tdse_observables")
tdse_apply_h = _fn("tdse_apply_h")
tdse_sync = _fn("tdse_sync")
tdse_fma_throughput = _fn("tdse_fma_throughput")
tdse_lanczos_expm = _fn("tdse_lanczos_expm")
tdse_set_small_grid_path = _fn("tdse_set_small_grid_path")
tdse_small_grid_path_used = _fn("tdse_small_grid_path_used")
tdse_set_persistent_path = _fn("tdse_set_persistent_path")
tdse_persistent_path_used = _fn("tdse_persistent_path_used")
tdse_launch_count = _fn("tdse_launch_count")
tdse_profile = _fn("tdse_profile")
tdse_profile_read = _fn("tdse_profile_read")
tdse_observables_noalloc = _fn("tdse_observables_noalloc")
TDSE_NOALLOC_MAX_LMAX = 255
tdse_batch_create = _fn("tdse_batch_create")
tdse_batch_destroy = _fn("tdse_batch_destroy")
tdse_batch_last_error = _fn("tdse_batch_last_error")
tdse_batch_set_stream = _fn("tdse_batch_set_stream")
tdse_batch_set_state = _fn("tdse_batch_set_state")
tdse_batch_get_state = _fn("tdse_batch_get_state")
tdse_batch_get_time = _fn("tdse_batch_get_time")
tdse_batch_set_time = _fn("tdse_batch_set_time")
tdse_batch_set_states = _fn("tdse_batch_set_states")
tdse_batch_get_states = _fn("tdse_batch_get_states")
tdse_batch_propagate = _fn("tdse_batch_propagate")
tdse_batch_propagate_io = _fn("tdse_batch_propagate_io")
tdse_batch_observables = _fn("tdse_batch_observables")
tdse_batch_dipole_series = _fn("tdse_batch_dipole_series")
tdse_batch_dipole_series_read = _fn("tdse_batch_dipole_series_read")
tdse_batch_propagate_imag = _fn("tdse_batch_propagate_imag")
tdse_batch_flux_setup = _fn("tdse_batch_flux_setup")
tdse_batch_flux_read = _fn("tdse_batch_flux_read")
tdse_batch_points = _fn("tdse_batch_points")
tdse_batch_launch_count = _fn("tdse_batch_launch_count")
tdse_batch_graph_steps = _fn("tdse_batch_graph_steps")
tdse_batch_profile = _fn("tdse_batch_profile")
tdse_batch_profile_read = _fn("tdse_batch_profile_read")
tdse_batch_autotune = _fn("tdse_batch_autotune")
tdse_batch_set_schedule = _fn("tdse_batch_set_schedule")
tdse_batch_get_schedule = _fn("tdse_batch_get_schedule")
tdse_server_autotune = _fn("tdse_server_autotune")
tdse_server_set_schedule = _fn("tdse_server_set_schedule")
tdse_server_instance_bytes = _fn("tdse_server_instance_bytes")
tdse_server_create = _fn("tdse_server_create")
tdse_server_destroy = _fn("tdse_server_destroy")
tdse_server_last_error = _fn("tdse_server_last_error")
tdse_server_set_stream = _fn("tdse_server_set_stream")
tdse_server_submit = _fn("tdse_server_submit")
tdse_server_step = _fn("tdse_server_step")
tdse_server_sync = _fn("tdse_server_sync")
tdse_server_poll = _fn("tdse_server_poll")
tdse_server_status = _fn("tdse_server_status")
tdse_server_observables = _fn("tdse_server_observables")
tdse_server_get_state = _fn("tdse_server_get_state")
tdse_server_release = _fn("tdse_server_release")
tdse_server_stats = _fn("tdse_server_stats")
tdse_server_profile = _fn("tdse_server_profile")
tdse_server_profile_read = _fn("tdse_server_profile_read")

KERNEL_KINDS = ["apply_h", "taylor_stage", "rk_stage", "norm", "lanczos_a", "lanczos_b",
                "lanczos_expm", "lanczos_combine", "observables", "dipole", "flux", "small_grid",
                "lanczos_persistent"]
