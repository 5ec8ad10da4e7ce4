"""ctypes binding of libmsm_gb300.so (include/msm_gb300.h): argument marshalling only.

The library is the product: every step of the method runs in its CUDA
kernels. If the shared library is missing this module raises; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmsm_gb300.so")

MSM_OK = 0
MSM_ERR_INVALID_ARG = 1
MSM_ERR_UNSUPPORTED = 2
MSM_ERR_CUDA = 3
MSM_ERR_NO_FORWARD = 4
MSM_ERR_CAPACITY = 5
MSM_DEV_OUT_OF_CELL = 1
MSM_DEV_NONFINITE = 2
MSM_DEV_NON_NEUTRAL = 4  # warning: a periodic system with a net charge (computed as defined)
MSM_DEV_CHECK = 8  # debug builds: an out-of-range index was caught (the access skipped)
MSM_DEV_ERRORS = MSM_DEV_OUT_OF_CELL | MSM_DEV_NONFINITE | MSM_DEV_CHECK
MSM_WANT_FORCES = 1
MSM_WANT_VIRIAL = 2

# every symbol include/msm_gb300.h declares
EXPORTS = [
    "msm_plan_create", "msm_plan_destroy", "msm_plan_get_info", "msm_plan_describe", "msm_plan_stencil",
    "msm_workspace_bytes", "msm_forward",
    "msm_backward", "msm_status", "msm_debug_offset", "msm_last_error", "msm_batch_create", "msm_batch_destroy",
    "msm_batch_workspace_bytes", "msm_batch_forward", "msm_batch_backward", "msm_batch_status", "msm_profile",
    "msm_profile_read", "msm_forward_noalloc", "msm_autotune", "msm_batch_autotune", "msm_batch_get_tuning",
    "msm_set_tuning", "msm_batch_set_tuning", "msm_field", "msm_batch_field", "msm_plan_set_cell", "msm_force_vjp",
    "msm_batch_force_vjp", "msm_potential_vjp", "msm_batch_potential_vjp", "msm_evaluate_host",
    "msm_set_level_method",
]
NOALLOC_SCRATCH_BYTES = 32 << 20
PHASES = ["bin", "short", "anterp", "restrict", "stencil", "prolong", "interp", "final", "virial", "bscale"]


class MsmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("msm error %d: %s" % (code, msg))
        self.code = code


class Params(C.Structure):
    _fields_ = [("cell", C.c_double * 9), ("pbc", C.c_int * 3), ("h", C.c_double), ("grid_override", C.c_int * 3),
                ("cutoff", C.c_double), ("order", C.c_int), ("levels", C.c_int), ("qi_mode", C.c_int),
                ("max_atoms", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("nlev", C.c_int), ("ncomp", C.c_int), ("M", C.c_int * 3), ("h1", C.c_double * 3),
                ("lo", (C.c_int * 3) * 20), ("n", (C.c_int * 3) * 20), ("R", C.c_int * 3), ("C", C.c_int * 3),
                ("nnbr", C.c_int * 3), ("stencil_kind", C.c_int * 20), ("anterp_tz", C.c_int),
                ("short_block", C.c_int), ("anterp_kind", C.c_int), ("level_method", C.c_int),
                ("spectral_ok", C.c_int)]


_lib = None
_vp = C.c_void_p


def load(path: str = None):
    """Load the shared library (built by build.py / __graft_entry__.build()). The
    environment variable MSM_GB300_LIB selects another build of it (the debug
    build with device-side index checks, libmsm_gb300_checks.so)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("MSM_GB300_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError("libmsm_gb300.so not found at %s: build it first (python -m paper_2510_05961_gb300.build)"
                          % path)
    L = C.CDLL(path)
    L.msm_last_error.restype = C.c_char_p
    L.msm_last_error.argtypes = []
    L.msm_plan_create.argtypes = [C.POINTER(Params), C.POINTER(_vp)]
    L.msm_plan_destroy.argtypes = [_vp]
    L.msm_plan_get_info.argtypes = [_vp, C.POINTER(PlanInfo)]
    L.msm_plan_describe.argtypes = [C.POINTER(Params), C.POINTER(PlanInfo)]
    L.msm_plan_stencil.argtypes = [C.POINTER(Params), C.c_int, C.c_int, _vp, C.c_size_t, C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]
    L.msm_workspace_bytes.argtypes = [_vp, C.POINTER(C.c_size_t)]
    L.msm_forward.argtypes = [_vp, _vp, C.c_size_t, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]
    L.msm_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.msm_status.argtypes = [_vp, _vp, _vp, C.POINTER(C.c_int)]
    L.msm_debug_offset.argtypes = [_vp, C.c_int, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    L.msm_batch_create.argtypes = [C.POINTER(Params), C.POINTER(C.c_int), C.c_int, C.POINTER(_vp)]
    L.msm_batch_destroy.argtypes = [_vp]
    L.msm_batch_workspace_bytes.argtypes = [_vp, C.POINTER(C.c_size_t)]
    L.msm_batch_forward.argtypes = [_vp, _vp, C.c_size_t, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]
    L.msm_batch_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.msm_batch_status.argtypes = [_vp, _vp, _vp, C.POINTER(C.c_int)]
    L.msm_field.argtypes = [_vp, _vp, _vp, _vp]
    L.msm_plan_set_cell.argtypes = [_vp, C.POINTER(C.c_double), _vp]
    L.msm_force_vjp.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.msm_batch_force_vjp.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.msm_potential_vjp.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.msm_evaluate_host.argtypes = [_vp, _vp, C.c_size_t, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.msm_batch_potential_vjp.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.msm_batch_field.argtypes = [_vp, _vp, _vp, _vp]
    L.msm_forward_noalloc.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp]
    L.msm_profile.argtypes = [_vp, C.c_int]
    L.msm_set_level_method.argtypes = [_vp, C.c_int]
    L.msm_autotune.argtypes = [_vp, _vp, C.c_size_t, C.c_int, _vp, _vp, _vp]
    L.msm_batch_autotune.argtypes = [_vp, _vp, C.c_size_t, _vp, _vp, _vp]
    L.msm_set_tuning.argtypes = [_vp, C.c_int, C.c_int]
    L.msm_batch_set_tuning.argtypes = [_vp, C.c_int, C.c_int]
    L.msm_batch_get_tuning.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.msm_profile_read.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    for name in EXPORTS:
        getattr(L, name).restype = C.c_int if name != "msm_last_error" else C.c_char_p
    _lib = L
    return L


def check(rc):
    if rc != MSM_OK:
        msg = load().msm_last_error()
        raise MsmError(rc, msg.decode() if msg else "")


def make_params(cell, pbc, h, cutoff, order, levels=0, grid_override=(0, 0, 0), max_atoms=0, qi_mode=0):
    P = Params()
    cell = list(cell)
    if len(cell) == 3:
        cell = [cell[0], 0, 0, 0, cell[1], 0, 0, 0, cell[2]]
    for i in range(9):
        P.cell[i] = float(cell[i])
    for d in range(3):
        P.pbc[d] = int(pbc[d])
        P.grid_override[d] = int(grid_override[d])
    P.h = float(h)
    P.cutoff = float(cutoff)
    P.order = int(order)
    P.levels = int(levels)
    P.qi_mode = int(qi_mode)
    P.max_atoms = int(max_atoms)
    return P
