"""ctypes declarations of the C-ABI in include/das.h.

Loads libdas_gb300.so from this package directory.  There is no fallback: if
the library is missing or cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdas_gb300.so")

DAS_OK, DAS_ERR_INVALID_ARG, DAS_ERR_CUDA, DAS_ERR_OOM, DAS_ERR_UNSUPPORTED, DAS_ERR_TIMEOUT = range(6)
DAS_TX_DIVERGING, DAS_TX_PLANE, DAS_TX_NONE = 0, 1, 2
DAS_SAMPLE_F32, DAS_SAMPLE_C64 = 0, 1
DAS_STORE_F32, DAS_STORE_F16, DAS_STORE_BF16, DAS_STORE_E4M3, DAS_STORE_E5M2 = 0, 1, 2, 3, 4

ERROR_NAMES = {DAS_ERR_INVALID_ARG: "invalid argument", DAS_ERR_CUDA: "CUDA error", DAS_ERR_OOM: "out of memory",
               DAS_ERR_UNSUPPORTED: "unsupported", DAS_ERR_TIMEOUT: "timeout"}

# Every symbol declared in include/das.h.
EXPORTS = ["das_plan_create", "das_plan_destroy", "das_plan_set_c", "das_plan_info", "das_plan_set_tuning",
           "das_forward", "das_forward_host", "das_adjoint", "das_grad_c", "das_count_active",
           "das_plan_enable_timing", "das_plan_timing", "das_last_error", "das_version", "das_grad_c_static",
           "das_plan_check", "das_batch_create", "das_batch_forward", "das_batch_set_tuning", "das_batch_info",
           "das_batch_destroy", "das_host_alloc", "das_host_free", "das_forward_host_many",
           "das_plan_set_wait_test"]


class Geometry(C.Structure):
    _fields_ = [("n_elements", C.c_int), ("positions", C.POINTER(C.c_double)),
                ("normals", C.POINTER(C.c_double)), ("t0_ref", C.c_double * 3)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("origin", C.c_double * 3),
                ("spacing", C.c_double * 3)]


class Tx(C.Structure):
    _fields_ = [("kind", C.c_int), ("vec", C.c_double * 3), ("w_tx", C.POINTER(C.c_float))]


class Options(C.Structure):
    _fields_ = [("n_samples", C.c_int), ("sample_type", C.c_int), ("storage", C.c_int),
                ("max_batch", C.c_int), ("t0_offset", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [("n_voxels", C.c_longlong), ("n_elements", C.c_int), ("n_transmits", C.c_int),
                ("n_samples", C.c_int), ("sample_type", C.c_int), ("storage", C.c_int), ("max_batch", C.c_int),
                ("device_bytes", C.c_longlong), ("c", C.c_double), ("kernel_launches", C.c_longlong),
                ("tc_mma_items", C.c_longlong), ("tc_mma_n", C.c_int)]


class Tuning(C.Structure):
    _fields_ = [("frames_per_thread", C.c_int), ("ctas_per_sm", C.c_int), ("staging", C.c_int),
                ("load_width", C.c_int), ("tensor_cores", C.c_int), ("tc_chain", C.c_int),
                ("voxels_per_thread", C.c_int), ("adjoint_rows", C.c_int), ("host_io", C.c_int)]


class DASError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded library (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2606_13259_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.das_plan_create.argtypes = [C.POINTER(vp), C.POINTER(Geometry), C.POINTER(Grid), C.POINTER(Tx), i, d, d,
                                      d, d, C.POINTER(Options)]
        L.das_plan_create.restype = i
        L.das_plan_destroy.argtypes = [vp]
        L.das_plan_destroy.restype = None
        L.das_plan_set_c.argtypes = [vp, d]
        L.das_plan_set_c.restype = i
        L.das_plan_info.argtypes = [vp, C.POINTER(PlanInfo)]
        L.das_plan_info.restype = i
        L.das_plan_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.das_plan_set_tuning.restype = i
        for name in ("das_forward", "das_forward_host", "das_adjoint"):
            getattr(L, name).argtypes = [vp, vp, vp, i, vp]
            getattr(L, name).restype = i
        L.das_forward_host_many.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), i, i, vp]
        L.das_forward_host_many.restype = i
        L.das_grad_c.argtypes = [vp, vp, vp, vp, i, vp]
        L.das_grad_c.restype = i
        L.das_grad_c_static.argtypes = [vp, vp, vp, vp, i, vp]
        L.das_grad_c_static.restype = i
        L.das_count_active.argtypes = [vp, C.POINTER(C.c_longlong), vp]
        L.das_count_active.restype = i
        L.das_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int), i]
        L.das_batch_create.restype = i
        L.das_batch_forward.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), vp]
        L.das_batch_forward.restype = i
        L.das_batch_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.das_batch_set_tuning.restype = i
        L.das_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.das_batch_info.restype = i
        L.das_batch_destroy.argtypes = [vp]
        L.das_batch_destroy.restype = None
        L.das_plan_check.argtypes = [vp, vp]
        L.das_plan_check.restype = i
        L.das_plan_set_wait_test.argtypes = [vp, C.c_longlong, i]
        L.das_plan_set_wait_test.restype = i
        L.das_plan_enable_timing.argtypes = [vp, i]
        L.das_plan_enable_timing.restype = i
        L.das_plan_timing.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
        L.das_plan_timing.restype = i
        L.das_last_error.argtypes = []
        L.das_last_error.restype = C.c_char_p
        L.das_version.argtypes = []
        L.das_version.restype = C.c_char_p
        L.das_host_alloc.argtypes = [C.c_size_t, C.POINTER(vp)]
        L.das_host_alloc.restype = i
        L.das_host_free.argtypes = [vp]
        L.das_host_free.restype = i
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != DAS_OK:
        raise DASError(rc, lib().das_last_error().decode(errors="replace"))
