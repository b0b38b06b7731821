"""ctypes declarations of libsmrt's C ABI (include/smrt.h). Loading fails loudly when the
library has not been built: there is no fallback implementation."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int8, c_size_t, c_uint, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsmrt.so")

LB_OK, LB_ERR_INVALID, LB_ERR_CUDA, LB_ERR_UNSTABLE, LB_ERR_TIMEOUT, LB_ERR_UNSUPPORTED, LB_ERR_NOMEM = range(7)
LB_F64, LB_F32, LB_F32_CONS64 = 0, 1, 2
LB_MOM_RHO, LB_MOM_U, LB_MOM_THETA, LB_MOM_SIGMA, LB_MOM_Q, LB_MOM_D = 0x1, 0x2, 0x4, 0x8, 0x10, 0x20
LB_MODEL_SMRT, LB_MODEL_ES_BGK = 0, 1
LB_HEALTH_UNSTABLE, LB_HEALTH_TIMEOUT = 0x1, 0x2


class LbLatticeDesc(ctypes.Structure):
    _fields_ = [("q", c_int), ("e", POINTER(c_int8)), ("w", POINTER(c_double)), ("c", c_double),
                ("degree", c_int), ("shift", c_int * 3)]


class LbGridDesc(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("batch", c_int),
                ("nx_per_instance", POINTER(c_int)), ("bc_x", c_int)]


class LbState(ctypes.Structure):
    _fields_ = [("rho", c_double), ("u", c_double * 3), ("theta", c_double)]


class LbSchedule(ctypes.Structure):
    _fields_ = [("tile_width", c_int), ("blocks_per_sm", c_int), ("persistent", c_int),
                ("tensor_cores", c_int), ("ms_per_step", c_double)]


# name -> (restype, argtypes); every symbol include/smrt.h declares
SIGNATURES = {
    "lb_init_lattice": (c_int, [POINTER(c_void_p), POINTER(LbLatticeDesc), POINTER(LbGridDesc), c_int, c_int, c_void_p]),
    "lb_set_relaxation": (c_int, [c_void_p, POINTER(c_double), c_int, c_double, POINTER(LbState), POINTER(LbState), c_int]),
    "lb_set_frame_shift": (c_int, [c_void_p, c_int, c_int]),
    "lb_set_collision_model": (c_int, [c_void_p, c_int, c_int, c_double]),
    "lb_hermite_convergence": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p, c_void_p, c_void_p]),
    "lb_fill_equilibrium": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lb_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "lb_moments": (c_int, [c_void_p, c_void_p, c_void_p, c_uint]),
    "lb_step_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lb_moments_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_uint, c_void_p]),
    "lb_step_adjoint_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "lb_poll_status": (c_int, [c_void_p, POINTER(c_uint)]),
    "lb_set_schedule": (c_int, [c_void_p, POINTER(LbSchedule)]),
    "lb_get_schedule": (c_int, [c_void_p, POINTER(LbSchedule)]),
    "lb_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_int, POINTER(LbSchedule)]),
    "lb_step_graph": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "lb_test_barrier_timeout": (c_int, [c_void_p, c_void_p, c_void_p]),
    "lb_cells": (c_size_t, [c_void_p]),
    "lb_plane_stride": (c_size_t, [c_void_p]),
    "lb_state_elems": (c_size_t, [c_void_p]),
    "lb_num_moment_rows": (c_int, [c_void_p, c_uint]),
    "lb_lattice_named": (c_int, [c_char_p, POINTER(c_int8), POINTER(c_double), POINTER(c_double), POINTER(c_int), POINTER(c_int), c_int]),
    "lb_rankine_hugoniot": (c_int, [c_double, c_double, c_double, c_double, POINTER(LbState), POINTER(LbState)]),
    "lb_shock_frame": (c_int, [c_double, c_double, c_double, c_double, POINTER(c_double), POINTER(c_int)]),
    "lb_shock_shift": (c_int, [c_double, c_double, c_double, c_double, POINTER(c_int)]),
    "lb_error_string": (c_char_p, [c_int]),
    "lb_destroy": (None, [c_void_p]),
}

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsmrt.so is not built ({LIB_PATH}); run "
                              "python -c 'import __graft_entry__ as g; g.build()'")
        try:  # share PyTorch's CUDA runtime when torch is present
            import torch  # noqa: F401
        except ImportError:
            pass
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib
