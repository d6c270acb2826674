"""GPU parity of the forward pass against the FP64 oracle (through the C-ABI).

Floating-point bars: relative L2 error <= 1e-5 for float32 storage (the
accuracy asked of the plain float32 form), <= 2e-3 for 16-bit storage (f16
and bf16), 5e-2 for E4M3; and beside each, the largest element-wise error
relative to the image peak (tests/parity.py).  Integer decisions (which terms
contribute) are compared exactly through the term count, on scenes whose
aperture tests have no near-ties.
"""
import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S
from parity import BAR, ELEM_F32_PAPER, assert_parity, rel_l2  # noqa: F401  (rel_l2 re-exported)

pytestmark = pytest.mark.gpu
MM = 1e-3
TOL_F32 = BAR["f32"]


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def run_forward(das, scene, y, storage="f32", fb=0):
    plan = das.Plan.from_scene(scene, storage=storage, max_batch=y.shape[0])
    if fb:
        plan.set_tuning(frames_per_thread=fb)
    x = plan.forward(y.cuda()).cpu().numpy().reshape(y.shape[0], -1)
    plan.close()
    return x


def test_small_rf_matches_oracle(das, oracle):
    """32^3 voxels, 256 elements, 1 diverging wave, RF f32, simulated speckle + points + noise."""
    sc = S.scene_small()
    y = S.frames(sc, 1, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0)
    x = run_forward(das, sc, y)
    ref = oracle.forward(sc, y.numpy())
    assert_parity(x, ref, TOL_F32, what="small RF")
    img = np.abs(x[0]).reshape(sc.nz, sc.ny, sc.nx)
    for ix, iy, iz in S.SMALL_POINTS:
        sub = img[iz - 2:iz + 3, iy - 2:iy + 3, ix - 2:ix + 3]
        assert np.unravel_index(np.argmax(sub), sub.shape) == (2, 2, 2)


def test_small_iq_matches_oracle(das, oracle):
    sc = S.scene_small_iq()
    y = S.frames(sc, 1, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0)
    x = run_forward(das, sc, y)
    ref = oracle.forward(sc, y.numpy())
    assert_parity(x, ref, TOL_F32, what="small IQ")


RAGGED = [
    # (iq, grid, elems, n_tx, f_number, K, kinds)
    (True, (13, 7, 9), (5, 3), 3, 1.0, 96, (S.TX_DIVERGING, S.TX_PLANE, S.TX_NONE)),
    (False, (9, 5, 6), (4, 4), 2, 0.0, 80, (S.TX_DIVERGING, S.TX_DIVERGING)),
    (True, (8, 4, 4), (3, 2), 2, 0.7, 56, (S.TX_PLANE, S.TX_DIVERGING)),
    (True, (17, 11, 5), (6, 5), 4, 1.3, 40, (S.TX_DIVERGING,) * 4),  # short K: many terms out of range
]


def ragged_scene(iq, grid, elems, n_tx, fnum, K, kinds):
    sc = S.scene_tiny(iq=iq, n=grid, elems=elems, n_tx=n_tx, f_number=fnum, K=K)
    vec = sc.tx_vec.copy()
    for q, k in enumerate(kinds):
        if k == S.TX_PLANE:
            a = 0.2 * (q - 1)
            vec[q] = [np.sin(a), 0.0, np.cos(a)]
    return sc.with_(tx_kind=np.array(kinds, np.int32), tx_vec=vec)


@pytest.mark.parametrize("case", range(len(RAGGED)))
@pytest.mark.parametrize("B", [1, 3, 7])
def test_ragged_tiles_transmit_kinds_and_batches(das, oracle, case, B):
    sc = ragged_scene(*RAGGED[case])
    y = S.random_channels(sc, B, seed=10 + case)
    x = run_forward(das, sc, y)
    ref = oracle.forward(sc, y.numpy())
    assert_parity(x, ref, TOL_F32, what=f"ragged case {case}, {B} frames")


@pytest.mark.parametrize("fb", [1, 2, 4, 8, 10, 12, 16, 20])
def test_frames_per_thread_variants(das, oracle, fb):
    """Every compiled frames-per-thread width gives the same image (padding of
    the last frame chunk included)."""
    sc = ragged_scene(*RAGGED[0])
    B = 21
    y = S.random_channels(sc, B, seed=5)
    x = run_forward(das, sc, y, fb=fb)
    ref = oracle.forward(sc, y.numpy())
    assert_parity(x, ref, TOL_F32, what=f"{fb} frames per thread")


@pytest.mark.parametrize("B,storage,tol", [(45, "f32", 1e-5), (130, "f32", 1e-5), (45, "f16", 2e-3),
                                           (130, "bf16", 2e-3)])
def test_large_batches_in_several_frame_chunks(das, oracle, B, storage, tol):
    """Batches of several frame chunks with a ragged last one (45 frames: 20 +
    20 + 5 with float32 rows) and a large batch (130 frames), default widths."""
    sc = ragged_scene(*RAGGED[0])
    y = S.random_channels(sc, B, seed=B + 100)
    x = run_forward(das, sc, y, storage=storage)
    e2, em = assert_parity(x, oracle.forward(sc, y.numpy()), tol, what=f"{B} frames {storage}")
    print(f"{B} frames, {storage}: relative L2 {e2:.3e}, element-wise {em:.3e}")


def test_transmit_weights(das, oracle):
    sc = ragged_scene(*RAGGED[0])
    rng = np.random.default_rng(2)
    sc = sc.with_(w_tx=rng.random((sc.Q, sc.N)).astype(np.float32))
    y = S.random_channels(sc, 2, seed=3)
    assert_parity(run_forward(das, sc, y), oracle.forward(sc, y.numpy()), TOL_F32, what="transmit weights")


def test_iq_without_demodulation_and_no_time_offset(das, oracle):
    sc = ragged_scene(*RAGGED[2]).with_(f_demod=0.0, t0_offset=False, K=128)
    y = S.random_channels(sc, 2, seed=4)
    assert_parity(run_forward(das, sc, y), oracle.forward(sc, y.numpy()), TOL_F32, what="no demodulation")


@pytest.mark.parametrize("name", ["small", "small_iq", "ragged0", "ragged3"])
def test_term_count_is_exact(das, oracle, name):
    sc = {"small": S.scene_small, "small_iq": S.scene_small_iq,
          "ragged0": lambda: ragged_scene(*RAGGED[0]), "ragged3": lambda: ragged_scene(*RAGGED[3])}[name]()
    assert oracle.count_near_ties(sc, 1e-5) == 0
    plan = das.Plan.from_scene(sc)
    assert plan.count_active() == oracle.count_active(sc)
    plan.close()


@pytest.mark.parametrize("storage,tol,iq", [("f16", 2e-3, False), ("f16", 2e-3, True), ("bf16", 2e-3, False),
                                            ("bf16", 2e-3, True), ("e4m3", 5e-2, True), ("e5m2", 1e-1, True)])
def test_16bit_storage(das, oracle, storage, tol, iq):
    """16-bit (and 8-bit E4M3 / E5M2) storage with a float32 scale per (transmit,
    element), float32 interpolation and sums."""
    sc = S.scene_small_iq() if iq else S.scene_small()
    y = S.frames(sc, 2, seed=1, n_speckle=2000, points=S.SMALL_POINTS, noise_db=30.0)
    x = run_forward(das, sc, y, storage=storage)
    ref = oracle.forward(sc, y.numpy())
    e2, em = assert_parity(x, ref, tol, what=f"{storage} iq={iq}")
    print(f"{storage} iq={iq}: relative L2 {e2:.3e}, element-wise {em:.3e}")


def test_paper_scale_sampled(das, oracle):
    """128^3 voxels x 1024 elements x 16 transmits, 20 IQ frames, in the launch
    configuration the benchmark times; compared on 96 sampled voxels."""
    sc = S.scene_paper()
    B = 20
    y = S.frames(sc, B, seed=2, n_speckle=20000, points=S.paper_points(sc), device="cuda")
    plan = das.Plan.from_scene(sc, max_batch=B)
    x = plan.forward(y).reshape(B, -1)
    rng = np.random.default_rng(0)
    vox = np.sort(rng.choice(sc.N, 96, replace=False))
    pts = [sc.voxel_index(*p) for p in S.paper_points(sc)]
    vox = np.concatenate([vox, pts])
    got = x[:, torch.as_tensor(vox, device="cuda")].cpu().numpy()
    ref = oracle.forward(sc, y.cpu().numpy(), voxels=vox)
    e2, em = assert_parity(got, ref, TOL_F32, ELEM_F32_PAPER, what="paper scale sampled")
    print(f"paper scale: relative L2 {e2:.3e}, element-wise {em:.3e} on {vox.size} voxels x {B} frames")
    plan.close()


def test_paper_scale_full_frames(das, oracle):
    """The benchmark's launch (128^3 voxels x 1024 elements x 16 transmits, 20
    IQ frames in one float32 call) against the oracle on every voxel of the
    first and the last frame of the chunk (2 x 2097152 voxels)."""
    sc = S.scene_paper()
    B = 20
    y = S.frames(sc, B, seed=2, n_speckle=20000, points=S.paper_points(sc), device="cuda")
    plan = das.Plan.from_scene(sc, max_batch=B)
    x = plan.forward(y).reshape(B, -1)
    plan.check()
    plan.close()
    frames = [0, B - 1]
    got = x[frames].cpu().numpy()
    ref = oracle.forward(sc, y[frames].cpu().numpy())
    e2, em = assert_parity(got, ref, TOL_F32, ELEM_F32_PAPER, what="paper scale, full frames")
    print(f"paper scale, frames {frames} in full: relative L2 {e2:.3e}, element-wise {em:.3e}")


def test_invalid_arguments_raise(das):
    sc = S.scene_tiny()
    plan = das.Plan.from_scene(sc, max_batch=2)
    y = S.random_channels(sc, 3, seed=0).cuda()
    with pytest.raises(ValueError):
        plan.forward(y)  # batch above max_batch
    with pytest.raises(TypeError):
        plan.forward(y[:1].real.contiguous())
    plan.close()
    with pytest.raises(das.DASError):
        das.Plan.from_scene(sc.with_(c=-1.0))


@pytest.mark.parametrize("staging,load_width", [(True, 0), (False, 0), (False, 128), (False, 256)])
@pytest.mark.parametrize("fb,storage", [(2, "f32"), (8, "f32"), (20, "f32"), (4, "f16"), (12, "bf16"), (16, "f16")])
def test_staged_and_global_sample_windows(das, oracle, staging, load_width, fb, storage):
    """Sample windows staged in shared memory by bulk copies, and rows read
    straight from global memory in column order (the default) or in row order
    with 128- or 256-bit loads, give the same image; the plan records no
    kernel-side failure."""
    sc = ragged_scene(*RAGGED[0])
    B = 23
    y = S.random_channels(sc, B, seed=8)
    plan = das.Plan.from_scene(sc, storage=storage, max_batch=B)
    plan.set_tuning(frames_per_thread=fb, staging=staging, load_width=load_width)
    x = plan.forward(y.cuda()).cpu().numpy().reshape(B, -1)
    plan.check()
    plan.close()
    ref = oracle.forward(sc, y.numpy())
    e2, em = assert_parity(x, ref, BAR[storage], what=f"fb {fb} {storage} staging={staging} width={load_width}")
    print(f"fb {fb} {storage} staging={staging} width={load_width}: relative L2 {e2:.3e}, element-wise {em:.3e}")


PAIR_SCENES = {
    # odd number of tiles along x (the last block holds one tile), three transmit kinds
    "ragged_odd_tiles": lambda: ragged_scene(*RAGGED[3]),
    # x spacing 0.3 mm: neighbours along x up to ~3 samples apart, so the
    # separate-rows branch of the pair kernel runs beside the shared-row one
    "wide_x_spacing": lambda: S.scene_tiny(iq=True, n=(21, 6, 9), elems=(5, 4), n_tx=3, f_number=0.8,
                                           K=160).with_(spacing=(0.3e-3, 0.1e-3, 0.1e-3)),
    # paper geometry, a crop with ragged tiles
    "paper_crop": lambda: S.scene_paper(512).with_(nx=40, ny=10, nz=9),
}


@pytest.mark.parametrize("name", sorted(PAIR_SCENES))
@pytest.mark.parametrize("B,fb", [(3, 4), (8, 8), (20, 20), (23, 12)])
def test_pair_kernel_matches_oracle_and_single_voxel_kernel(das, oracle, name, B, fb):
    """Two x-adjacent voxels per thread sharing rows (the float32 IQ default)
    against the oracle and against the one-voxel-per-thread kernel."""
    sc = PAIR_SCENES[name]()
    y = S.random_channels(sc, B, seed=90 + fb)
    ref = oracle.forward(sc, y.numpy())
    out = {}
    for vpt in (1, 2):
        plan = das.Plan.from_scene(sc, max_batch=B)
        plan.set_tuning(frames_per_thread=fb, voxels_per_thread=vpt)
        out[vpt] = plan.forward(y.cuda()).cpu().numpy().reshape(B, -1)
        plan.check()
        plan.close()
        assert_parity(out[vpt], ref, TOL_F32, what=f"{name}, {vpt} voxels per thread, fb {fb}")
    assert_parity(out[2], out[1], TOL_F32, what=f"{name}: pair kernel against the one-voxel kernel")


def test_staged_paper_tile_geometry_small_batch(das, oracle):
    """Paper geometry cropped to 32 x 24 x 20 voxels (ragged tiles), 4 frames:
    staged windows against the oracle on every voxel."""
    sc = S.scene_paper(512).with_(nx=32, ny=24, nz=20)
    B = 4
    y = S.frames(sc, B, seed=3, n_speckle=3000, points=[], device="cuda")
    plan = das.Plan.from_scene(sc, max_batch=B)
    x = plan.forward(y).reshape(B, -1).cpu().numpy()
    plan.check()
    plan.close()
    ref = oracle.forward(sc, y.cpu().numpy())
    assert_parity(x, ref, TOL_F32, what="staged paper geometry")


@pytest.mark.parametrize("kind", ["huge_pages", "pinned", "pageable"])
def test_forward_host_matches_device_call(das, kind):
    """Host buffers in, host buffers out (copies split across the plan's copy
    streams): the same image as the device call, for huge-page buffers from
    das_host_alloc, torch-pinned and plain pageable memory."""
    sc = ragged_scene(*RAGGED[0])
    B = 5
    y = S.random_channels(sc, B, seed=12)
    plan = das.Plan.from_scene(sc, max_batch=B)
    ref = plan.forward(y.cuda()).cpu()
    if kind == "huge_pages":
        yh, xh = das.host_empty(y.shape, y.dtype), das.host_empty(ref.shape, ref.dtype)
        assert yh.is_pinned() and xh.is_pinned()
    elif kind == "pinned":
        yh, xh = torch.empty(y.shape, dtype=y.dtype).pin_memory(), torch.empty(ref.shape, dtype=ref.dtype).pin_memory()
    else:
        yh, xh = torch.empty(y.shape, dtype=y.dtype), torch.empty(ref.shape, dtype=ref.dtype)
    yh.copy_(y)
    plan.forward_host(yh, xh)
    plan.close()
    assert torch.equal(xh, ref)


@pytest.mark.parametrize("kind", ["huge_pages", "pinned"])
def test_direct_host_io_matches_device_call(das, kind):
    """host_io = 2: the kernels read the channel data from page-locked host
    memory and write the image there directly (no copies, no staging), for
    one call and for a sequence; bit-identical to the device call.  A pageable
    buffer is either refused before any launch or, where the GPU reaches host
    memory through the host's page tables (this platform), read directly with
    the same result."""
    sc = ragged_scene(*RAGGED[0])
    B = 5
    ys = [S.random_channels(sc, B, seed=140 + i) for i in range(3)]
    plan = das.Plan.from_scene(sc, max_batch=B)
    refs = [plan.forward(y.cuda()).cpu() for y in ys]
    plan.set_tuning(host_io=2)
    alloc = (lambda shape, dt: das.host_empty(shape, dt)) if kind == "huge_pages" else \
        (lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory())
    yh = [alloc(y.shape, y.dtype) for y in ys]
    for h, y in zip(yh, ys):
        h.copy_(y)
    xh = alloc(refs[0].shape, refs[0].dtype)
    plan.forward_host(yh[0], xh)
    assert torch.equal(xh, refs[0])
    outs = plan.forward_host_many(yh)
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    pageable = torch.empty(ys[0].shape, dtype=ys[0].dtype)
    pageable.copy_(ys[0])
    xh.zero_()
    try:
        plan.forward_host(pageable, xh)
        assert torch.equal(xh, refs[0])
    except das.DASError:
        pass
    plan.check()
    plan.close()


@pytest.mark.parametrize("n_batches,B", [(1, 5), (2, 5), (5, 3)])
def test_forward_host_many_matches_device_calls(das, n_batches, B):
    """A sequence of host batches with copies overlapped with the forward
    passes (two staging slots): every image equals the device call's, for
    sequences shorter than, equal to and longer than the two slots, and a
    batch smaller than the plan's largest."""
    sc = ragged_scene(*RAGGED[0])
    plan = das.Plan.from_scene(sc, max_batch=5)
    ys = [S.random_channels(sc, B, seed=40 + i) for i in range(n_batches)]
    refs = [plan.forward(y.cuda()).cpu() for y in ys]
    yh = []
    for y in ys:
        h = das.host_empty(y.shape, y.dtype)
        h.copy_(y)
        yh.append(h)
    outs = plan.forward_host_many(yh)
    # the same input buffer twice in one sequence
    again = plan.forward_host_many([yh[0], yh[0]])
    plan.check()
    plan.close()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    assert torch.equal(again[0], refs[0]) and torch.equal(again[1], refs[0])


def test_host_empty_large_block_round_trip(das):
    """A block larger than one huge page survives a device round trip."""
    n = 3 * (1 << 27) + 12345  # ~ 1.5 GB of uint8 spread over several huge pages
    h = das.host_empty((n,), torch.uint8)
    h[:: 1 << 20] = 7
    d = h.cuda()
    back = das.host_empty((n,), torch.uint8)
    back.copy_(d)
    assert torch.equal(back[:: 1 << 20], h[:: 1 << 20])


DEGENERATE = {
    # one voxel, one element, one transmit, the smallest K
    "single": dict(n=(1, 1, 1), elems=(1, 1), n_tx=1, K=2, f_number=0.0),
    "single_k64": dict(n=(1, 1, 1), elems=(1, 1), n_tx=1, K=64, f_number=0.0),
    # a thin line of voxels and a line array, full aperture
    "line": dict(n=(17, 1, 1), elems=(7, 1), n_tx=1, K=64, f_number=0.0),
}


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("name", sorted(DEGENERATE))
def test_degenerate_shapes(das, oracle, name, tc):
    """1 voxel / 1 element / 1 transmit, K = 2 (no term lies in range), thin
    grids: CUDA-core and tensor-core paths against the oracle."""
    sc = S.scene_tiny(iq=True, **DEGENERATE[name])
    y = S.random_channels(sc, 3, seed=31)
    plan = das.Plan.from_scene(sc, storage="f16" if tc else "f32", max_batch=3)
    if tc:
        plan.set_tuning(tensor_cores=True)
    x = plan.forward(y.cuda()).cpu().numpy().reshape(3, -1)
    plan.check()
    plan.close()
    ref = oracle.forward(sc, y.numpy())
    if np.linalg.norm(ref) == 0.0:
        assert np.count_nonzero(x) == 0
    else:
        assert_parity(x, ref, BAR["f16"] if tc else TOL_F32, what=name)


@pytest.mark.parametrize("tc", [False, True])
def test_most_transmits_a_plan_takes(das, oracle, tc):
    """128 transmits (the most a plan takes; a mix of diverging waves, plane
    waves and none) on a ragged grid: shared-memory tables of 128 x 128
    transmit rests per tile, and on the tensor cores lists of 16384 pairs per
    element block, cut at 4096 sub-items."""
    sc = S.scene_tiny(iq=True, n=(11, 6, 5), elems=(4, 3), n_tx=128, f_number=1.0, K=96)
    kinds = np.array([(q % 3) for q in range(128)], np.int32)
    vec = sc.tx_vec.copy()
    for q in range(128):
        if kinds[q] == S.TX_PLANE:
            a = 0.3 * np.sin(q)
            vec[q] = [np.sin(a), 0.0, np.cos(a)]
        elif kinds[q] == S.TX_NONE:
            vec[q] = [0.0, 0.0, 0.0]
    sc = sc.with_(tx_kind=kinds, tx_vec=vec)
    y = S.random_channels(sc, 3, seed=150)
    plan = das.Plan.from_scene(sc, storage="f16" if tc else "f32", max_batch=3)
    if tc:
        plan.set_tuning(tensor_cores=True)
    x = plan.forward(y.cuda()).cpu().numpy().reshape(3, -1)
    plan.check()
    plan.close()
    assert_parity(x, oracle.forward(sc, y.numpy()), BAR["f16"] if tc else TOL_F32, what="128 transmits")


@pytest.mark.parametrize("tc", [False, True])
def test_no_voxel_inside_any_aperture(das, oracle, tc):
    """Voxels at the depth of the array (z = 0 plane), f-number 1: every term
    is outside the aperture and the image is exactly zero."""
    sc = S.scene_tiny(iq=True, n=(9, 5, 3), elems=(3, 3), n_tx=2, K=64, f_number=1.0)
    sc = sc.with_(origin=(sc.origin[0], sc.origin[1], -0.5e-3))
    y = S.random_channels(sc, 2, seed=32)
    ref = oracle.forward(sc, y.numpy())
    assert np.count_nonzero(ref) == 0
    plan = das.Plan.from_scene(sc, storage="f16" if tc else "f32", max_batch=2)
    if tc:
        plan.set_tuning(tensor_cores=True)
    x = plan.forward(y.cuda()).cpu().numpy()
    plan.check()
    plan.close()
    assert np.count_nonzero(x) == 0
