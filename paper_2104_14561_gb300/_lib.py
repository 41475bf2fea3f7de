"""ctypes declarations of the C ABI in include/fk.h.

The library is the only compute path: if it cannot be loaded this module
raises, and nothing falls back to CPU code.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfk_gb300.so")

FK_OK = 0
STATUS = {0: "FK_OK", 1: "FK_ERR_INVALID_ARG", 2: "FK_ERR_UNSUPPORTED", 3: "FK_ERR_OOM",
          4: "FK_ERR_CUDA", 5: "FK_ERR_TIMEOUT", 6: "FK_ERR_DEVICE"}

FK_FP32, FK_FP64 = 0, 1
FK_PATH_MATRIX_FREE, FK_PATH_CSR = 0, 1
FK_CONST_DRIFT, FK_CELLULAR_FLOW, FK_PAPER_CELLULAR, FK_RUNAWAY_3D = 0, 1, 2, 3
FK_RUNAWAY_QUENCH_3D = 4
FK_ALL_FACES_ABSORBING = 0x3F
FK_PERIODIC_X = 0x3C

# every symbol include/fk.h declares
EXPORTS = ("fk_plan_create", "fk_plan_destroy", "fk_plan_get_info", "fk_gauss_hermite",
           "fk_solve", "fk_solve_host", "fk_march", "fk_solve_horizons", "fk_solve_batched",
           "fk_adjoint",
           "fk_status_string", "fk_last_device_error", "fk_solve_static",
           "fk_static_last_device_error", "fk_runaway_quench_params", "fk_measure_fma_rate",
           "fk_adjoint_kernel_times")


class FkError(RuntimeError):
    def __init__(self, call: str, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{call} failed: {STATUS.get(status, status)}{': ' + detail if detail else ''}")


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("axis", ctypes.POINTER(ctypes.c_double) * 3)]


class Region(ctypes.Structure):
    _fields_ = [("absorbing_faces", ctypes.c_uint)]


class Coeffs(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("p", ctypes.c_double * 16)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_interior", ctypes.c_int64),
                ("dim", ctypes.c_int), ("q_per_dim", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("precision", ctypes.c_int), ("path", ctypes.c_int),
                ("halo", ctypes.c_int * 3), ("tile", ctypes.c_int * 3),
                ("reach_cells", ctypes.c_double * 3), ("csr_nnz", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("window_rows", ctypes.c_int),
                ("step_kernel", ctypes.c_int), ("batch_mode", ctypes.c_int),
                ("adjoint_kernel", ctypes.c_int), ("periodic_x", ctypes.c_int),
                ("nonuniform", ctypes.c_int), ("march_mode", ctypes.c_int),
                ("nodes_per_thread", ctypes.c_int)]


_lib = None


def load(build_if_missing: bool = False):
    """Load libfk_gb300.so (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if build_if_missing:
            from .build import build
            build()
        else:
            raise ImportError(f"{LIB_PATH} is missing: run paper_2104_14561_gb300.build.build() "
                              "(nvcc, sm_103a) first; there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    st = ctypes.c_int
    lib.fk_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Grid), ctypes.POINTER(Region),
                                   ctypes.POINTER(Coeffs), ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.fk_plan_create.restype = st
    lib.fk_plan_destroy.argtypes = [vp]
    lib.fk_plan_destroy.restype = st
    lib.fk_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.fk_plan_get_info.restype = st
    lib.fk_gauss_hermite.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.fk_gauss_hermite.restype = st
    lib.fk_runaway_quench_params.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_double)]
    lib.fk_runaway_quench_params.restype = st
    lib.fk_solve.argtypes = [vp, vp, vp, vp, ctypes.c_int, vp]
    lib.fk_solve.restype = st
    lib.fk_solve_host.argtypes = [vp, vp, vp, vp]
    lib.fk_solve_host.restype = st
    lib.fk_march.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.fk_march.restype = st
    lib.fk_solve_horizons.argtypes = [vp, vp, vp, vp]
    lib.fk_solve_horizons.restype = st
    lib.fk_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp), vp]
    lib.fk_solve_batched.restype = st
    lib.fk_adjoint.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, vp]
    lib.fk_adjoint.restype = st
    lib.fk_status_string.argtypes = [st]
    lib.fk_status_string.restype = ctypes.c_char_p
    lib.fk_last_device_error.argtypes = [vp]
    lib.fk_last_device_error.restype = st
    lib.fk_static_last_device_error.argtypes = []
    lib.fk_static_last_device_error.restype = st
    lib.fk_measure_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double), vp]
    lib.fk_measure_fma_rate.restype = st
    lib.fk_adjoint_kernel_times.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_int)]
    lib.fk_adjoint_kernel_times.restype = st
    _lib = lib
    return lib


def check(call: str, status: int):
    if status != FK_OK:
        detail = ""
        if _lib is not None:
            detail = _lib.fk_status_string(status).decode()
        raise FkError(call, status, detail)
