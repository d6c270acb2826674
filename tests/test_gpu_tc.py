"""GPU parity of the tensor-core forward path (tcgen05 tile contraction, Sec. 3.4)
against the FP64 oracle, through the C-ABI.

The path stores samples and interpolation weights as 16-bit values and sums
in float32 (tensor memory), so it is held to the 16-bit bar: relative L2
error <= 2e-3 with f16 and with bf16 storage, and the same bound on the
largest element-wise error relative to the image peak (tests/parity.py).
Every case also checks that no kernel-side failure was recorded (bounded
waits, and terms falling outside the window the kernel bounded for them).
"""
import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S
from parity import BAR, assert_parity

from test_gpu_forward import RAGGED, ragged_scene

pytestmark = pytest.mark.gpu
TOL = {"f16": BAR["f16"], "bf16": BAR["bf16"]}


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def tc_forward(das, scene, y, storage="f16", ctas_per_sm=0, tc_chain=0):
    plan = das.Plan.from_scene(scene, storage=storage, max_batch=y.shape[0])
    plan.set_tuning(tensor_cores=True, ctas_per_sm=ctas_per_sm, tc_chain=tc_chain)
    x = plan.forward(y if y.is_cuda else y.cuda())
    plan.check()
    plan.close()
    return x.reshape(y.shape[0], -1)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_small_iq_scene(das, oracle, storage):
    """32^3 voxels, 256 elements, IQ: windows span up to four 15-row sub-items."""
    sc = S.scene_small_iq()
    y = S.frames(sc, 3, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0)
    x = tc_forward(das, sc, y, storage).cpu().numpy()
    e2, em = assert_parity(x, oracle.forward(sc, y.numpy()), TOL[storage], what=f"tensor cores {storage}")
    print(f"tensor cores {storage}: relative L2 {e2:.3e}, element-wise {em:.3e}")


@pytest.mark.parametrize("case", [0, 2, 3])
@pytest.mark.parametrize("B", [1, 5, 21])
def test_ragged_tiles_and_transmit_kinds(das, oracle, case, B):
    """Partial tiles, diverging / plane / no transmit, short K (terms out of range)."""
    sc = ragged_scene(*RAGGED[case])
    y = S.random_channels(sc, B, seed=20 + case)
    x = tc_forward(das, sc, y).cpu().numpy()
    assert_parity(x, oracle.forward(sc, y.numpy()), TOL["f16"], what=f"ragged case {case}, {B} frames")


@pytest.mark.parametrize("B,ctas", [(16, 0), (128, 0), (130, 0), (128, 2), (130, 2), (112, 2), (20, 3), (48, 4),
                                    (100, 3)])
def test_mma_widths_and_frame_chunks(das, oracle, B, ctas):
    """N = 32 and the largest N = 256 (128 frames), and two frame chunks (130
    frames); with two CTAs per SM at most 112 frames per chunk (128 frames:
    two chunks of 64, N = 128; 112 frames: one chunk, N = 224); with three or
    four CTAs per SM (one builder group each) at most 48 frames per chunk
    (100 frames: three chunks of 34, N = 80)."""
    sc = ragged_scene(*RAGGED[0])
    y = S.random_channels(sc, B, seed=B)
    x = tc_forward(das, sc, y, ctas_per_sm=ctas).cpu().numpy()
    assert_parity(x, oracle.forward(sc, y.numpy()), TOL["f16"], what=f"{B} frames, {ctas} CTAs per SM")


@pytest.mark.parametrize("chain,ctas,B", [(-1, 0, 3), (1, 0, 3), (1, 1, 3), (300, 0, 3), (1, 0, 130)])
def test_accumulation_chains(das, oracle, chain, ctas, B):
    """D added into the image at every list end (chain 1), after a few lists
    (300), or once per tile (-1); two and four builder groups; two frame chunks."""
    sc = S.scene_small_iq()
    y = S.frames(sc, B, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0)
    x = tc_forward(das, sc, y, ctas_per_sm=ctas, tc_chain=chain).cpu().numpy()
    e2, em = assert_parity(x, oracle.forward(sc, y.numpy()), TOL["f16"], what=f"chain {chain}")
    print(f"chain {chain}, ctas/SM {ctas or 'auto'}, {B} frames: relative L2 {e2:.3e}, element-wise {em:.3e}")


def test_transmit_weights_and_one_cta_per_sm(das, oracle):
    sc = ragged_scene(*RAGGED[0])
    rng = np.random.default_rng(2)
    sc = sc.with_(w_tx=rng.random((sc.Q, sc.N)).astype(np.float32))
    y = S.random_channels(sc, 4, seed=3)
    x = tc_forward(das, sc, y, ctas_per_sm=1).cpu().numpy()
    assert_parity(x, oracle.forward(sc, y.numpy()), TOL["f16"], what="transmit weights")


def test_without_demodulation(das, oracle):
    sc = ragged_scene(*RAGGED[2]).with_(f_demod=0.0, t0_offset=False, K=128)
    y = S.random_channels(sc, 2, seed=4)
    x = tc_forward(das, sc, y).cpu().numpy()
    assert_parity(x, oracle.forward(sc, y.numpy()), TOL["f16"], what="no demodulation")


def test_matches_cuda_core_path(das):
    """Same plan, same data: the tensor-core image against the float32 CUDA-core image."""
    sc = S.scene_small_iq()
    y = S.frames(sc, 4, seed=5, n_speckle=2000, points=S.SMALL_POINTS, device="cuda")
    ref_plan = das.Plan.from_scene(sc, max_batch=4)
    ref = ref_plan.forward(y).reshape(4, -1)
    ref_plan.close()
    x = tc_forward(das, sc, y)
    assert_parity(x.cpu().numpy(), ref.cpu().numpy(), TOL["f16"], what="against the CUDA-core image")


def test_paper_scale_sampled(das, oracle):
    """128^3 voxels x 1024 elements x 16 transmits, 20 IQ frames (the benchmark's
    workload and launch), 96 sampled voxels plus the ten point targets."""
    sc = S.scene_paper()
    B = 20
    y = S.frames(sc, B, seed=2, n_speckle=20000, points=S.paper_points(sc), device="cuda")
    x = tc_forward(das, sc, y)
    rng = np.random.default_rng(0)
    vox = np.concatenate([np.sort(rng.choice(sc.N, 96, replace=False)),
                          [sc.voxel_index(*p) for p in S.paper_points(sc)]])
    got = x[:, torch.as_tensor(vox, device="cuda")].cpu().numpy()
    e2, em = assert_parity(got, oracle.forward(sc, y.cpu().numpy(), voxels=vox), TOL["f16"], what="paper scale")
    print(f"paper scale, tensor cores: relative L2 {e2:.3e}, element-wise {em:.3e}")


def test_paper_scale_full_frames(das, oracle):
    """The benchmark's tensor-core launch (paper workload, 20 IQ frames, f16)
    against the oracle on every voxel of the first and the last frame."""
    sc = S.scene_paper()
    B = 20
    y = S.frames(sc, B, seed=2, n_speckle=20000, points=S.paper_points(sc), device="cuda")
    x = tc_forward(das, sc, y)
    frames = [0, B - 1]
    got = x[frames].cpu().numpy()
    ref = oracle.forward(sc, y[frames].cpu().numpy())
    e2, em = assert_parity(got, ref, TOL["f16"], what="paper scale, tensor cores, full frames")
    print(f"paper scale, tensor cores, frames {frames} in full: relative L2 {e2:.3e}, element-wise {em:.3e}")


def test_paper_scale_gain_at_point_targets(das, oracle):
    """The tensor core's float32 accumulation loses a little of the running
    sum at every step, a gain deficit proportional to the chain length (about
    7e-4 at the point targets of the paper workload with one chain per tile).
    With the default chains of 1024 sub-items the gain at the ten point
    targets stays within 1.5e-4 of the oracle's."""
    sc = S.scene_paper()
    B = 20
    y = S.frames(sc, B, seed=2, n_speckle=20000, points=S.paper_points(sc), device="cuda")
    pts = np.array([sc.voxel_index(*p) for p in S.paper_points(sc)])
    ref = oracle.forward(sc, y.cpu().numpy(), voxels=pts)
    gains = {}
    for chain in (0, -1):
        got = tc_forward(das, sc, y, tc_chain=chain)[:, torch.as_tensor(pts, device="cuda")].cpu().numpy()
        gains[chain] = float(np.real(np.vdot(ref, got)) / np.vdot(ref, ref).real) - 1.0
    print(f"gain error at the point targets: chains of 1024 {gains[0]:+.2e}, one chain {gains[-1]:+.2e}")
    assert abs(gains[0]) <= 1.5e-4


def test_table1_configuration_sampled(das, oracle):
    """The Table 1 configuration (128^3 voxels at lambda/2, 1024 elements at
    lambda pitch, one plane wave, K = 256) with 128 frames: N = 256."""
    sc = S.scene_table1()
    B = 128
    y = S.frames(sc, B, seed=4, n_speckle=20000, points=S.paper_points(sc), device="cuda")
    x = tc_forward(das, sc, y)
    rng = np.random.default_rng(1)
    vox = np.concatenate([np.sort(rng.choice(sc.N, 48, replace=False)),
                          [sc.voxel_index(*p) for p in S.paper_points(sc)]])
    got = x[:, torch.as_tensor(vox, device="cuda")].cpu().numpy()
    e2, em = assert_parity(got, oracle.forward(sc, y.cpu().numpy(), voxels=vox), TOL["f16"], what="Table 1")
    print(f"Table 1 configuration, tensor cores: relative L2 {e2:.3e}, element-wise {em:.3e}")


def test_tensor_cores_need_16bit_iq(das):
    with pytest.raises(das.DASError):
        das.Plan.from_scene(S.scene_tiny(), storage="f32").set_tuning(tensor_cores=True)
    with pytest.raises(das.DASError):
        das.Plan.from_scene(S.scene_tiny(iq=False), storage="f16").set_tuning(tensor_cores=True)
