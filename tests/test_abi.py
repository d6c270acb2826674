"""The C-ABI library: it loads, exports every function include/das.h declares,
and rejects invalid arguments before touching the GPU (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_13259_gb300 import _lib
    from paper_2606_13259_gb300 import build as B

    B.build()
    return _lib


def declared_functions():
    text = open(os.path.join(ROOT, "include", "das.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(das_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree(lib):
    assert declared_functions() == sorted(lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    L = C.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name
    assert lib.lib().das_version().startswith(b"das-gb300")


def _args(lib, **over):
    pos = np.zeros((4, 3))
    pos[:, 0] = np.arange(4) * 3e-4
    geom = lib.Geometry()
    geom.n_elements = over.get("M", 4)
    geom.positions = pos.ctypes.data_as(C.POINTER(C.c_double))
    geom.normals = None
    grid = lib.Grid()
    grid.nx, grid.ny, grid.nz = over.get("grid", (4, 4, 4))
    grid.origin = (C.c_double * 3)(0, 0, 5e-3)
    grid.spacing = (C.c_double * 3)(*over.get("spacing", (1e-4, 1e-4, 1e-4)))
    tx = (lib.Tx * 1)()
    tx[0].kind = over.get("kind", 0)
    tx[0].vec = (C.c_double * 3)(*over.get("vec", (0, 0, -1e-2)))
    opt = lib.Options()
    opt.n_samples = over.get("K", 64)
    opt.sample_type = over.get("sample_type", 1)
    opt.storage = over.get("storage", 0)
    opt.max_batch = over.get("max_batch", 1)
    opt.t0_offset = 1
    return pos, geom, grid, tx, opt


@pytest.mark.parametrize("bad", [
    {"M": 0}, {"grid": (0, 4, 4)}, {"spacing": (1e-4, -1e-4, 1e-4)}, {"kind": 7}, {"K": 1},
    {"sample_type": 5}, {"storage": 9}, {"max_batch": 0}, {"kind": 1, "vec": (0.0, 0.0, 2.0)},
    {"c": -1.0}, {"fs": 0.0}, {"f_demod_rf": True}, {"n_tx": 0}, {"n_tx": 500},
])
def test_invalid_plan_arguments_rejected_before_gpu(lib, bad):
    pos, geom, grid, tx, opt = _args(lib, **bad)
    L = lib.lib()
    c = bad.get("c", 1540.0)
    fs = bad.get("fs", 15e6)
    fd = 7.5e6
    if bad.get("f_demod_rf"):
        opt.sample_type = 0
    n_tx = bad.get("n_tx", 1)
    h = C.c_void_p()
    rc = L.das_plan_create(C.byref(h), C.byref(geom), C.byref(grid), tx, n_tx, c, fs, fd, 1.0, C.byref(opt))
    assert rc in (lib.DAS_ERR_INVALID_ARG, lib.DAS_ERR_UNSUPPORTED)
    assert h.value is None
    assert len(L.das_last_error()) > 0


def test_null_arguments_rejected(lib):
    L = lib.lib()
    assert L.das_plan_create(None, None, None, None, 1, 1540.0, 1e7, 0.0, 1.0, None) == lib.DAS_ERR_INVALID_ARG
    assert L.das_forward(None, None, None, 1, None) == lib.DAS_ERR_INVALID_ARG
    assert L.das_adjoint(None, None, None, 1, None) == lib.DAS_ERR_INVALID_ARG
    assert L.das_grad_c(None, None, None, None, 1, None) == lib.DAS_ERR_INVALID_ARG
    assert L.das_plan_set_c(None, 1500.0) == lib.DAS_ERR_INVALID_ARG
    assert L.das_forward_host(None, None, None, 1, None) == lib.DAS_ERR_INVALID_ARG
    assert L.das_forward_host_many(None, None, None, 2, 1, None) == lib.DAS_ERR_INVALID_ARG
    L.das_plan_destroy(None)


def test_host_allocator_arguments(lib):
    """das_host_alloc / das_host_free reject bad arguments; without a GPU the
    registration fails cleanly (with one, the block is returned and freed)."""
    L = lib.lib()
    ptr = C.c_void_p()
    assert L.das_host_alloc(C.c_size_t(0), C.byref(ptr)) == lib.DAS_ERR_INVALID_ARG
    assert L.das_host_alloc(C.c_size_t(1 << 20), None) == lib.DAS_ERR_INVALID_ARG
    assert L.das_host_free(None) == lib.DAS_OK
    junk = (C.c_char * 64)()
    assert L.das_host_free(C.cast(junk, C.c_void_p)) == lib.DAS_ERR_INVALID_ARG
    rc = L.das_host_alloc(C.c_size_t(1 << 20), C.byref(ptr))
    if rc == lib.DAS_OK:
        assert ptr.value and ptr.value % 64 == 0
        assert L.das_host_free(ptr) == lib.DAS_OK
    else:
        assert rc == lib.DAS_ERR_CUDA and not ptr.value
