"""Failure handling of the pipelined kernels, made to happen on purpose and
read back on the host (no GPU fault: each kernel gives up a bounded wait,
records it in the plan's error word, drains its copies and MMAs in flight and
leaves; das_plan_check reports DAS_ERR_TIMEOUT).

* A wait that runs out: das_plan_set_wait_test makes the first CTA wait on a
  shared-memory barrier that nothing arrives on, with a 2 ms limit (the
  tensor-core kernel's MMA-issuing thread; warp 1 of the staged kernel).
* A work list too short for an item: a sample span of ~1.5e5 rows inside one
  voxel tile needs ~10^4 sixteen-row windows, more than the 4096 one list holds.

After each failure the same plan (hook off) and a fresh plan match the FP64
oracle again.
"""
import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S
from parity import BAR, assert_parity

from test_gpu_forward import RAGGED, ragged_scene

pytestmark = pytest.mark.gpu
LIMIT_NS = 2_000_000


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def expect_timeout(das, plan):
    with pytest.raises(das.DASError) as e:
        plan.check()
    assert e.value.code == das._lib.DAS_ERR_TIMEOUT
    plan.check()  # the record was cleared


def test_tensor_core_wait_runs_out(das, oracle):
    sc = S.scene_small_iq()
    y = S.frames(sc, 3, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0).cuda()
    ref = oracle.forward(sc, y.cpu().numpy())
    plan = das.Plan.from_scene(sc, storage="f16", max_batch=3)
    plan.set_tuning(tensor_cores=True)
    plan.set_wait_test(LIMIT_NS, probe=True)
    plan.forward(y)
    expect_timeout(das, plan)
    plan.set_wait_test(0, probe=False)
    x = plan.forward(y).reshape(3, -1)
    plan.check()
    plan.close()
    assert_parity(x.cpu().numpy(), ref, BAR["f16"], what="same plan after the expired wait")
    fresh = das.Plan.from_scene(sc, storage="f16", max_batch=3)
    fresh.set_tuning(tensor_cores=True)
    x = fresh.forward(y).reshape(3, -1)
    fresh.check()
    fresh.close()
    assert_parity(x.cpu().numpy(), ref, BAR["f16"], what="fresh plan after the expired wait")


def test_staged_wait_runs_out(das, oracle):
    sc = ragged_scene(*RAGGED[0])
    B = 8
    y = S.random_channels(sc, B, seed=70).cuda()
    ref = oracle.forward(sc, y.cpu().numpy())
    plan = das.Plan.from_scene(sc, max_batch=B)
    plan.set_tuning(frames_per_thread=8, staging=True)
    plan.set_wait_test(LIMIT_NS, probe=True)
    plan.forward(y)
    expect_timeout(das, plan)
    plan.set_wait_test(0, probe=False)
    x = plan.forward(y).reshape(B, -1)
    plan.check()
    plan.close()
    assert_parity(x.cpu().numpy(), ref, BAR["f32"], what="staged kernel after the expired wait")


def test_tensor_core_work_list_truncation(das, oracle):
    """One 8 x 4 x 4 voxel tile 1.0-1.3 mm deep above one element, a diverging
    wave from 5 mm behind it, full aperture, fs = 4e11 Hz (a = fs / c = 2.6e8
    samples per metre): the delays of the tile span a (0.3 mm transmit +
    0.3 mm receive) = 1.6e5 rows, about 10^4 windows of 15 rows."""
    sc = S.scene_tiny(iq=True, n=(8, 4, 4), elems=(1, 1), n_tx=1, f_number=0.0, K=700_000)
    sc = sc.with_(fs=4e11, tx_vec=np.array([[0.0, 0.0, -5e-3]]))
    y = S.random_channels(sc, 1, seed=71).cuda()
    plan = das.Plan.from_scene(sc, storage="f16", max_batch=1)
    plan.set_tuning(tensor_cores=True)
    plan.forward(y)
    expect_timeout(das, plan)
    plan.close()
    # a plan of ordinary span on the same path afterwards
    sc2 = S.scene_small_iq()
    y2 = S.frames(sc2, 2, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0).cuda()
    p2 = das.Plan.from_scene(sc2, storage="f16", max_batch=2)
    p2.set_tuning(tensor_cores=True)
    x = p2.forward(y2).reshape(2, -1)
    p2.check()
    p2.close()
    assert_parity(x.cpu().numpy(), oracle.forward(sc2, y2.cpu().numpy()), BAR["f16"], what="after truncation")
