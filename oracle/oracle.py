"""ctypes wrapper of the FP64 CPU oracle (das_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The product path never imports it.

`build()` compiles das_oracle.c with gcc + OpenMP into liboracle.so next to
this file.  Functions take a `Scene` (the plain-data description from the
input-generator module) and numpy arrays, and return numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "das_oracle.c")
LIB = os.environ.get("DAS_ORACLE_LIB") or os.path.join(HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, gcc, OpenMP)."""
    if os.environ.get("DAS_ORACLE_LIB"):
        return LIB
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "das_oracle.h"))):
        tmp = LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("origin", C.c_double * 3), ("spacing", C.c_double * 3),
        ("M", C.c_int), ("elem_pos", C.POINTER(C.c_double)), ("elem_normal", C.POINTER(C.c_double)),
        ("Q", C.c_int), ("tx_kind", C.POINTER(C.c_int)), ("tx_vec", C.POINTER(C.c_double)),
        ("w_tx", C.POINTER(C.c_double)), ("t0_ref", C.c_double * 3), ("t0_offset", C.c_int),
        ("c", C.c_double), ("fs", C.c_double), ("f_demod", C.c_double), ("f_number", C.c_double),
        ("K", C.c_int), ("iq", C.c_int),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        P = C.POINTER(Problem)
        dp, fp, lp = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_long)
        lib.oracle_forward.argtypes = [P, fp, C.c_int, lp, C.c_long, dp]
        lib.oracle_forward_f64.argtypes = [P, dp, C.c_int, lp, C.c_long, dp]
        lib.oracle_adjoint.argtypes = [P, dp, C.c_int, lp, C.c_long, dp]
        lib.oracle_grad_c.argtypes = [P, fp, dp, C.c_int, lp, C.c_long]
        lib.oracle_grad_c.restype = C.c_double
        lib.oracle_count_active.argtypes = [P]
        lib.oracle_count_active.restype = C.c_longlong
        lib.oracle_count_near_ties.argtypes = [P, C.c_double]
        lib.oracle_count_near_ties.restype = C.c_longlong
        lib.oracle_num_threads.restype = C.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


class _Prob:
    """Keeps the numpy buffers alive while the C struct points into them."""

    def __init__(self, scene, c=None):
        self.pos = np.ascontiguousarray(scene.elem_pos, dtype=np.float64)
        self.nrm = np.ascontiguousarray(scene.elem_normal, dtype=np.float64)
        self.kind = np.ascontiguousarray(scene.tx_kind, dtype=np.int32)
        self.vec = np.ascontiguousarray(scene.tx_vec, dtype=np.float64)
        self.wtx = None if scene.w_tx is None else np.ascontiguousarray(scene.w_tx, dtype=np.float64)
        s = Problem()
        s.nx, s.ny, s.nz = scene.nx, scene.ny, scene.nz
        s.origin = (C.c_double * 3)(*scene.origin)
        s.spacing = (C.c_double * 3)(*scene.spacing)
        s.M = self.pos.shape[0]
        s.elem_pos = self.pos.ctypes.data_as(C.POINTER(C.c_double))
        s.elem_normal = self.nrm.ctypes.data_as(C.POINTER(C.c_double))
        s.Q = self.vec.shape[0]
        s.tx_kind = self.kind.ctypes.data_as(C.POINTER(C.c_int))
        s.tx_vec = self.vec.ctypes.data_as(C.POINTER(C.c_double))
        s.w_tx = self.wtx.ctypes.data_as(C.POINTER(C.c_double)) if self.wtx is not None else None
        s.t0_ref = (C.c_double * 3)(*scene.t0_ref)
        s.t0_offset = int(bool(scene.t0_offset))
        s.c = float(scene.c if c is None else c)
        s.fs, s.f_demod, s.f_number = float(scene.fs), float(scene.f_demod), float(scene.f_number)
        s.K, s.iq = int(scene.K), int(bool(scene.iq))
        self.s = s

    def ref(self):
        return C.byref(self.s)


def _channels_f32(scene, y) -> np.ndarray:
    """Channel data as a contiguous float32 array ([..., 2] interleaved for IQ)."""
    a = np.asarray(y)
    if scene.iq:
        a = np.ascontiguousarray(a, dtype=np.complex64).view(np.float32)
    else:
        a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def _voxels(voxels):
    if voxels is None:
        return None, None, 0
    v = np.ascontiguousarray(np.asarray(voxels, dtype=np.int64))
    return v, v.ctypes.data_as(C.POINTER(C.c_long)), v.size


def forward(scene, y, voxels=None, c=None) -> np.ndarray:
    """Eq. 2 in FP64: y [B][Q][M][K] (float32 / complex64) -> x [B][nv] complex128."""
    lib = _load()
    y = np.asarray(y)
    B = y.shape[0]
    yf = _channels_f32(scene, y)
    v, vp, nv = _voxels(voxels)
    nv = scene.N if v is None else nv
    x = np.zeros((B, nv), dtype=np.complex128)
    p = _Prob(scene, c)
    lib.oracle_forward(p.ref(), yf.ctypes.data_as(C.POINTER(C.c_float)), B, vp, nv,
                       x.ctypes.data_as(C.POINTER(C.c_double)))
    return x


def forward_f64(scene, y, voxels=None, c=None) -> np.ndarray:
    """Eq. 2 in FP64 on double-precision channel data."""
    lib = _load()
    y = np.asarray(y)
    B = y.shape[0]
    if scene.iq:
        yd = np.ascontiguousarray(y.astype(np.complex128)).view(np.float64)
    else:
        yd = np.ascontiguousarray(y.real if np.iscomplexobj(y) else y, dtype=np.float64)
    v, vp, nv = _voxels(voxels)
    nv = scene.N if v is None else nv
    x = np.zeros((B, nv), dtype=np.complex128)
    p = _Prob(scene, c)
    lib.oracle_forward_f64(p.ref(), yd.ctypes.data_as(C.POINTER(C.c_double)), B, vp, nv,
                           x.ctypes.data_as(C.POINTER(C.c_double)))
    return x


def adjoint(scene, x, rows=None, c=None) -> np.ndarray:
    """DAS^H in FP64: x [B][N] complex -> y [B][nrows][K] complex128 (rows = q*M + m)."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    B = x.shape[0]
    r, rp, nr = _voxels(rows)
    nr = scene.Q * scene.M if r is None else nr
    y = np.zeros((B, nr, scene.K), dtype=np.complex128)
    p = _Prob(scene, c)
    lib.oracle_adjoint(p.ref(), x.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)), B, rp, nr,
                       y.ctypes.data_as(C.POINTER(C.c_double)))
    return y


def grad_c(scene, y, gx, voxels=None, c=None) -> float:
    """Re sum conj(gx) * dx/dc in FP64 (gx [B][nv] complex)."""
    lib = _load()
    y = np.asarray(y)
    B = y.shape[0]
    yf = _channels_f32(scene, y)
    g = np.ascontiguousarray(np.asarray(gx, dtype=np.complex128))
    v, vp, nv = _voxels(voxels)
    nv = scene.N if v is None else nv
    p = _Prob(scene, c)
    return float(lib.oracle_grad_c(p.ref(), yf.ctypes.data_as(C.POINTER(C.c_float)),
                                   g.view(np.float64).ctypes.data_as(C.POINTER(C.c_double)), B, vp, nv))


def count_active(scene, c=None) -> int:
    return int(_load().oracle_count_active(_Prob(scene, c).ref()))


def count_near_ties(scene, rel: float = 1e-5) -> int:
    return int(_load().oracle_count_near_ties(_Prob(scene).ref(), rel))


def loss_and_cotangent(x: np.ndarray):
    """L = -sum|x|^4 / (sum|x|^2)^2 and 2 dL/d conj(x) (the cotangent that
    makes dL/dc = Re sum conj(g) dx/dc)."""
    x = np.asarray(x, dtype=np.complex128)
    a2 = np.abs(x) ** 2
    s2, s4 = a2.sum(), (a2 * a2).sum()
    L = -s4 / s2 ** 2
    g = 2.0 * (-2.0 * x * (a2 * s2 - s4) / s2 ** 3)
    return float(L), g
