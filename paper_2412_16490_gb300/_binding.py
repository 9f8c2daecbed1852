"""ctypes binding of the C ABI in ``include/bodex.h``.

Argument marshalling only: every computation happens in the CUDA library.
The functions keep the ABI's names; device arrays are passed as raw
pointers taken from torch CUDA tensors, streams as ``cudaStream_t`` handles.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

c_float_p = C.POINTER(C.c_float)
c_int_p = C.POINTER(C.c_int32)

BODEX_OK = 0
BODEX_ERR_INVALID = 1
BODEX_ERR_CUDA = 2
BODEX_ERR_OOM = 3
BODEX_ERR_INFEASIBLE = 4
BODEX_ERR_TIMEOUT = 5
BODEX_ERR_NOT_CONVERGED = 6
ST_NONFINITE = 1
ST_NOT_CONVERGED = 2
ST_DEGENERATE_NORMAL = 4
ST_POLISHED = 8
QP_ADMM, QP_EXACT = 0, 1

# Every symbol include/bodex.h declares (checked by the CPU test-suite).
ENERGY_QP, ENERGY_DFC = 0, 1
CONE_PYRAMID, CONE_ELLIPTIC = 0, 1

EXPORTS = (
    "bodex_hand_create", "bodex_hand_destroy", "bodex_object_create", "bodex_object_destroy",
    "bodex_object_gravity_centre", "bodex_fk_contacts", "bodex_qp_solve_batch", "bodex_state_create",
    "bodex_state_destroy", "bodex_state_set_pose", "bodex_state_get_pose", "bodex_state_get_adam",
    "bodex_state_get_residual", "bodex_step_multi", "bodex_step_tile",
    "bodex_energy_grad", "bodex_energy_adjoint", "bodex_step", "bodex_refine", "bodex_contact_metrics", "bodex_squeeze_pose", "bodex_step_noalloc", "bodex_sync", "bodex_last_error", "bodex_version",
)


class bodex_hand_desc(C.Structure):
    _fields_ = [("n_joints", C.c_int), ("n_contacts", C.c_int), ("parent", c_int_p), ("offset", c_float_p),
                ("axis", c_float_p), ("qmin", c_float_p), ("qmax", c_float_p), ("contact_link", c_int_p),
                ("contact_local", c_float_p), ("contact_radius", C.c_float), ("n_tip_samples", C.c_int),
                ("tip_samples", c_float_p), ("n_spheres", C.c_int), ("sphere_link", c_int_p),
                ("sphere_local", c_float_p), ("sphere_radius", c_float_p)]


class bodex_object_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("center", C.c_float * 3), ("radius", C.c_float), ("n", C.c_int),
                ("h", C.c_float), ("origin", C.c_float * 3), ("values", c_float_p)]


class bodex_qp_params(C.Structure):
    _fields_ = [("mu", C.c_float), ("beta", C.c_float), ("gamma", C.c_float), ("rho", C.c_float),
                ("sigma", C.c_float), ("alpha", C.c_float), ("eps_abs", C.c_float), ("eps_reg", C.c_float),
                ("max_iter", C.c_int), ("check_every", C.c_int), ("warm", C.c_int), ("strict", C.c_int),
                ("cone", C.c_int), ("adaptive_rho", C.c_int), ("polish", C.c_int), ("solver", C.c_int)]


class bodex_energy_params(C.Structure):
    _fields_ = [("w_q", C.c_float), ("w_d", C.c_float), ("delta", C.c_float), ("kind", C.c_int),
                ("w_pen", C.c_float), ("w_self", C.c_float), ("w_lim", C.c_float), ("eta_pen", C.c_float),
                ("eta_lim", C.c_float)]


class bodex_step_params(C.Structure):
    _fields_ = [("lr_t", C.c_float), ("lr_r", C.c_float), ("b1", C.c_float), ("b2", C.c_float),
                ("adam_eps", C.c_float), ("energy", bodex_energy_params), ("qp", bodex_qp_params),
                ("grasps_per_cta", C.c_int), ("work_pulling", C.c_int)]


class bodex_job(C.Structure):
    _fields_ = [("hand", C.c_void_p), ("obj", C.c_void_p), ("state", C.c_void_p), ("T", C.c_void_p),
                ("s", C.c_int), ("n_steps", C.c_int), ("E_last", C.c_void_p), ("status", C.c_void_p)]


BODEX_MAX_JOBS = 64


_lib = None


class BodexError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bodex error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbodex.so (building it with nvcc when missing or stale).

    There is no CPU fallback: if the library cannot be built or loaded this
    raises."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library {_build.LIB} is missing; run paper_2412_16490_gb300._build.build()")
    L = C.CDLL(_build.LIB)
    v = C.c_void_p
    vp = C.POINTER(C.c_void_p)
    sig = {
        "bodex_hand_create": [C.POINTER(bodex_hand_desc), vp],
        "bodex_hand_destroy": [v],
        "bodex_object_create": [C.POINTER(bodex_object_desc), v, vp],
        "bodex_object_destroy": [v],
        "bodex_object_gravity_centre": [v, c_float_p],
        "bodex_fk_contacts": [v, v, v, C.c_int, v, v, v, v, v, v, v, v],
        "bodex_qp_solve_batch": [v, C.c_int, C.c_int, v, C.c_int, C.POINTER(bodex_qp_params), v, v, v, v, v, v,
                                 v, v],
        "bodex_state_create": [v, C.c_int, C.c_int, vp],
        "bodex_state_destroy": [v],
        "bodex_state_set_pose": [v, v, v],
        "bodex_state_get_pose": [v, v, v],
        "bodex_state_get_adam": [v, v, v, C.POINTER(C.c_int), v],
        "bodex_state_get_residual": [v, v, v],
        "bodex_step_multi": [C.POINTER(bodex_job), C.c_int, C.POINTER(bodex_step_params), v],
        "bodex_step_tile": [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)],
        "bodex_energy_grad": [v, v, v, C.c_int, v, C.c_int, C.POINTER(bodex_step_params), v, v, v, v, v, v, v],
        "bodex_energy_adjoint": [v, v, v, C.c_int, v, C.c_int, C.POINTER(bodex_step_params), v, v, v, v, v],
        "bodex_step": [v, v, v, v, C.c_int, C.c_int, C.POINTER(bodex_step_params), v, v, v],
        "bodex_refine": [v, v, v, v, C.c_int, C.c_float, C.c_float, C.POINTER(bodex_step_params), v, v, v, v],
        "bodex_contact_metrics": [v, v, v, C.c_int, v, v, v],
        "bodex_squeeze_pose": [v, v, C.c_int, C.c_int, v, v],
        "bodex_step_noalloc": [v, v, v, C.c_int, v, C.c_int, C.c_int, C.POINTER(bodex_step_params), v, v, v],
        "bodex_sync": [v],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.bodex_last_error.restype = C.c_char_p
    L.bodex_last_error.argtypes = []
    L.bodex_version.restype = C.c_char_p
    L.bodex_version.argtypes = []
    _lib = L
    return L


def check(code: int):
    if code != BODEX_OK:
        raise BodexError(code, load(False).bodex_last_error().decode())
    return code
