"""Batched form: several uneven plans and all their frames in one persistent
launch replayed from a CUDA graph, checked against the FP64 oracle and
against single-plan calls; the autotuner's choice keeps the result."""
import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S
from parity import BAR, assert_parity, rel_l2
from test_gpu_forward import RAGGED, ragged_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def three_scenes():
    return [ragged_scene(*RAGGED[0]), ragged_scene(*RAGGED[3]),
            S.scene_tiny(iq=True, n=(20, 9, 12), elems=(7, 4), n_tx=5, f_number=1.0, K=72)]


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_matches_oracle_and_replays(das, oracle, storage):
    scenes = three_scenes()
    frames = [3, 2, 5]
    ys = [S.random_channels(sc, f, seed=60 + i).cuda() for i, (sc, f) in enumerate(zip(scenes, frames))]
    plans = [das.Plan.from_scene(sc, storage=storage, max_batch=f) for sc, f in zip(scenes, frames)]
    batch = das.Batch(plans, frames)
    tol = BAR[storage]
    for rep in range(2):  # capture, then replay
        outs = batch.forward(ys)
        for sc, y, x, p in zip(scenes, ys, outs, plans):
            ref = oracle.forward(sc, y.cpu().numpy())
            assert_parity(x.reshape(x.shape[0], -1).cpu().numpy(), ref, tol, what=f"{sc.name} {storage}")
            p.check()
    # single-plan calls give the same images
    for p, y, x in zip(plans, ys, outs):
        single = p.forward(y)
        assert rel_l2(x.cpu().numpy(), single.cpu().numpy()) <= 1e-6
    # new data pointers: a new graph
    ys2 = [y.clone() * 2 for y in ys]
    outs2 = batch.forward(ys2)
    for x, x2 in zip(outs, outs2):
        assert rel_l2(x2.cpu().numpy(), 2 * x.cpu().numpy()) <= 1e-6
    info = batch.info()
    assert info["kernels_per_launch"] == len(plans) * (1 if storage == "f32" else 2) + 1
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("fb,ctas", [(4, 1), (8, 2), (24, 0), (12, 3)])
def test_batch_tuning_variants_agree(das, fb, ctas):
    scenes = three_scenes()
    frames = [5, 7, 3]
    ys = [S.random_channels(sc, f, seed=70 + i).cuda() for i, (sc, f) in enumerate(zip(scenes, frames))]
    plans = [das.Plan.from_scene(sc, storage="f16", max_batch=f) for sc, f in zip(scenes, frames)]
    batch = das.Batch(plans, frames)
    ref = [x.clone() for x in batch.forward(ys)]
    batch.set_tuning(fb, ctas)
    got = batch.forward(ys)
    for a, b in zip(ref, got):
        assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) <= 1e-6
    batch.close()
    for p in plans:
        p.close()


def test_batched_workload_plans_sampled(das, oracle):
    """The three plans of the batched workload (64^3 / 512 el / 4 tx, 128x128x96 /
    1024 el / 9 tx, 128^3 / 1024 el / 16 tx), FP16 IQ, 2 frames each."""
    scenes = S.scenes_batched()
    frames = [2, 2, 2]
    ys = [S.frames(sc, f, seed=80 + i, n_speckle=4000, points=S.paper_points(sc), device="cuda")
          for i, (sc, f) in enumerate(zip(scenes, frames))]
    plans = [das.Plan.from_scene(sc, storage="f16", max_batch=f) for sc, f in zip(scenes, frames)]
    batch = das.Batch(plans, frames)
    outs = batch.forward(ys)
    rng = np.random.default_rng(1)
    for sc, y, x, p in zip(scenes, ys, outs, plans):
        vox = np.concatenate([rng.choice(sc.N, 48, replace=False), [sc.voxel_index(*q) for q in S.paper_points(sc)]])
        got = x.reshape(x.shape[0], -1)[:, torch.as_tensor(vox, device="cuda")].cpu().numpy()
        ref = oracle.forward(sc, y.cpu().numpy(), voxels=vox)
        e2, em = assert_parity(got, ref, BAR["f16"], what=sc.name)
        print(f"{sc.name}: f16 relative L2 {e2:.2e}, element-wise {em:.2e}")
        p.check()
    batch.close()
    for p in plans:
        p.close()


def test_autotuner_choice_keeps_result(das, tmp_path, monkeypatch):
    from paper_2606_13259_gb300 import autotune

    monkeypatch.setenv("DAS_TUNING_CACHE", str(tmp_path / "tuning.json"))
    scenes = three_scenes()
    frames = [4, 4, 4]
    ys = [S.random_channels(sc, f, seed=90 + i).cuda() for i, (sc, f) in enumerate(zip(scenes, frames))]
    plans = [das.Plan.from_scene(sc, storage="f16", max_batch=f) for sc, f in zip(scenes, frames)]
    batch = das.Batch(plans, frames)
    ref = [x.clone() for x in batch.forward(ys)]
    outs = [torch.empty_like(x) for x in ref]
    res = autotune.tune_batch(batch, ys, outs, ctas=(0, 2), reps=1)
    assert not res["cached"] and res["frames_per_thread"] in autotune.F16_FB
    res2 = autotune.tune_batch(batch, ys, outs)
    assert res2["cached"] and res2["frames_per_thread"] == res["frames_per_thread"]
    for a, b in zip(ref, batch.forward(ys)):
        assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) <= 1e-6
    pr = autotune.tune_plan(plans[0], ys[0], outs[0], reps=1)
    assert pr["tensor_cores"] or pr["frames_per_thread"] >= 1
    # whichever kernel won, the plan's image stays within the 16-bit bar
    x = plans[0].forward(ys[0])
    plans[0].check()
    assert_parity(x.cpu().numpy(), ref[0].cpu().numpy(), BAR["f16"], what="tuned plan")
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("tc_plans", [(True, False, False), (True, True, True)])
def test_batch_with_tensor_core_plans(das, oracle, tc_plans):
    """Plans whose own tuning selects the tensor cores run as their own
    launches inside the batch's graph, the others in the persistent launch
    (all three on the tensor cores: no persistent launch at all); every image
    against the oracle at the 16-bit bar, on capture and on replay."""
    scenes = three_scenes()
    frames = [3, 2, 5]
    ys = [S.random_channels(sc, f, seed=110 + i).cuda() for i, (sc, f) in enumerate(zip(scenes, frames))]
    plans = [das.Plan.from_scene(sc, storage="f16", max_batch=f) for sc, f in zip(scenes, frames)]
    for p, tc in zip(plans, tc_plans):
        p.set_tuning(tensor_cores=tc)
    batch = das.Batch(plans, frames)
    n_cc = sum(1 for tc in tc_plans if not tc)
    for rep in range(2):  # capture, then replay
        outs = batch.forward(ys)
        for sc, y, x, p in zip(scenes, ys, outs, plans):
            assert_parity(x.reshape(x.shape[0], -1).cpu().numpy(), oracle.forward(sc, y.cpu().numpy()), BAR["f16"],
                          what=f"{sc.name}, tensor cores {p.info()['tc_mma_n'] > 0}")
            p.check()
    info = batch.info()
    assert (info["work_items"] > 0) == (n_cc > 0)
    batch.close()
    for p in plans:
        p.close()
