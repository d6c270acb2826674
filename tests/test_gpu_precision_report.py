"""Error of every storage form and forward path against the FP64 oracle:
relative L2 and max-abs error (the largest |x - x_ref| over the largest
|x_ref|, i.e. relative to the image peak), printed as one table row each and
held to the bars of the forms (float32 1e-5, f16 2e-3, bf16 2e-2, E4M3 5e-2,
relative L2).

Workloads: the small scene (32^3 voxels, 256 elements, RF and IQ, 2 frames),
and sampled voxels of the paper workload (128^3 x 1024 x 16, 20 IQ frames)
and of the Table 1 configuration (128 frames).
"""
import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S

pytestmark = pytest.mark.gpu
BAR = {"f32": 1e-5, "f16": 2e-3, "bf16": 2e-2, "e4m3": 5e-2}


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def errors(x, ref):
    x, ref = np.asarray(x), np.asarray(ref)
    rel = float(np.linalg.norm(x - ref) / np.linalg.norm(ref))
    mx = float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))
    return rel, mx


def run(das, sc, y, storage, tc, voxels=None):
    B = y.shape[0]
    plan = das.Plan.from_scene(sc, storage=storage, max_batch=B)
    if tc:
        plan.set_tuning(tensor_cores=True)
    x = plan.forward(y if y.is_cuda else y.cuda()).reshape(B, -1)
    plan.check()
    plan.close()
    if voxels is not None:
        x = x[:, torch.as_tensor(voxels, device=x.device)]
    return x.cpu().numpy()


CASES = [("small RF", False, "f32", False), ("small RF", False, "f16", False), ("small RF", False, "bf16", False),
         ("small IQ", True, "f32", False), ("small IQ", True, "f16", False), ("small IQ", True, "bf16", False),
         ("small IQ", True, "e4m3", False), ("small IQ", True, "f16", True), ("small IQ", True, "bf16", True)]


@pytest.mark.parametrize("name,iq,storage,tc", CASES)
def test_small_scene_errors(das, oracle, name, iq, storage, tc):
    sc = S.scene_small_iq() if iq else S.scene_small()
    y = S.frames(sc, 2, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0)
    rel, mx = errors(run(das, sc, y, storage, tc), oracle.forward(sc, y.numpy()))
    print(f"\n| {name} | {'tensor cores' if tc else 'CUDA cores'} | {storage} | {rel:.2e} | {mx:.2e} |")
    assert rel <= BAR[storage]


@pytest.mark.parametrize("workload,storage,tc", [("paper", "f32", False), ("paper", "f16", False),
                                                 ("paper", "f16", True), ("table1", "f16", True)])
def test_full_size_sampled_errors(das, oracle, workload, storage, tc):
    sc = S.scene_paper() if workload == "paper" else S.scene_table1()
    B = 20 if workload == "paper" else 128
    y = S.frames(sc, B, seed=2, n_speckle=20000, points=S.paper_points(sc), device="cuda")
    rng = np.random.default_rng(3)
    vox = np.concatenate([np.sort(rng.choice(sc.N, 64, replace=False)),
                          [sc.voxel_index(*p) for p in S.paper_points(sc)]])
    x = run(das, sc, y, storage, tc, voxels=vox)
    rel, mx = errors(x, oracle.forward(sc, y.cpu().numpy(), voxels=vox))
    print(f"\n| {workload} (sampled) | {'tensor cores' if tc else 'CUDA cores'} | {storage} | {rel:.2e} | {mx:.2e} |")
    assert rel <= BAR[storage]
