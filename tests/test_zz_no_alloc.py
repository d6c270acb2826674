"""das_grad_c_static: the sound-speed derivative with its scratch in a fixed
array inside the library, for callers that cannot allocate device memory
where they need the derivative.  Called through the C-ABI twice in a row and
compared with das_grad_c; oversized problems are refused before any launch.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S

pytestmark = pytest.mark.gpu
TOL = 1e-4  # the relative tolerance the derivative tests use against the oracle


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def _call(das, fn, plan, y, g, out, B):
    from paper_2606_13259_gb300 import _lib

    rc = getattr(_lib.lib(), fn)(plan._h, C.c_void_p(y.data_ptr()), C.c_void_p(g.data_ptr()),
                                C.c_void_p(out.data_ptr()), B, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(rc)
    torch.cuda.synchronize()
    return float(out.cpu())


@pytest.mark.parametrize("iq,B", [(True, 3), (False, 1), (True, 21)])
def test_static_scratch_matches_das_grad_c(das, iq, B):
    """On a fresh plan the static call comes first (its first-use set-up is
    what runs), then again with the device memory recorded around it: neither
    the driver's free memory, nor torch's allocator, nor the plan's own device
    bytes change.  Both results equal das_grad_c's within the derivative
    tests' tolerance."""
    sc = S.scene_tiny(iq=iq, n=(13, 7, 9), elems=(5, 3), n_tx=3, f_number=1.0, K=96)
    y = S.random_channels(sc, B, seed=50).cuda()
    g = S.random_image(sc, B, seed=51)
    g = (g if iq else g.real.contiguous()).cuda()
    plan = das.Plan.from_scene(sc, max_batch=B)
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    first = _call(das, "das_grad_c_static", plan, y, g, out, B)
    torch.cuda.synchronize()
    free0, torch0, plan0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), plan.info()["device_bytes"]
    second = _call(das, "das_grad_c_static", plan, y, g, out, B)
    free1, torch1, plan1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), plan.info()["device_bytes"]
    assert (free1, torch1, plan1) == (free0, torch0, plan0)
    ref = _call(das, "das_grad_c", plan, y, g, out, B)
    assert abs(first - ref) <= TOL * abs(ref)
    assert abs(second - ref) <= TOL * abs(ref)
    plan.close()


def test_static_scratch_refuses_oversized_problem(das):
    """512 x 512 x 64 voxels are 131072 tiles; any frames-per-thread value of
    20 or less cuts 41 frames into at least 3 chunks, and 3 x 131072 partial
    sums are more than the 262144 the static array holds.  The refusal comes
    from the host before any launch, so the data pointers only need to be
    aligned device pointers."""
    from paper_2606_13259_gb300 import _lib

    sc = S.scene_tiny(iq=True, n=(512, 512, 64), elems=(2, 1), n_tx=1, f_number=1.0, K=16)
    B = 41
    plan = das.Plan.from_scene(sc, max_batch=B)
    y = torch.zeros(16, dtype=torch.complex64, device="cuda")
    g = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    rc = _lib.lib().das_grad_c_static(plan._h, C.c_void_p(y.data_ptr()), C.c_void_p(g.data_ptr()),
                                      C.c_void_p(out.data_ptr()), B, None)
    assert rc == _lib.DAS_ERR_UNSUPPORTED
    assert b"static scratch" in _lib.lib().das_last_error()
    plan.close()
