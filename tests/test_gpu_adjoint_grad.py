"""GPU parity of the adjoint (image -> channel data) and of the sound-speed
derivative against the FP64 oracle, through the C-ABI, plus the autograd
wrapper."""
import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S
from parity import assert_parity, rel_l2
from test_gpu_forward import RAGGED, ragged_scene

pytestmark = pytest.mark.gpu
TOL_F32 = 1e-5


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def image_like(sc, B, seed):
    x = S.random_image(sc, B, seed)
    return x if sc.iq else x.real.contiguous()


@pytest.mark.parametrize("case", range(len(RAGGED)))
@pytest.mark.parametrize("B", [1, 2, 5])
def test_adjoint_matches_oracle(das, oracle, case, B):
    sc = ragged_scene(*RAGGED[case])
    x = image_like(sc, B, seed=20 + case)
    plan = das.Plan.from_scene(sc, max_batch=B)
    y = plan.adjoint(x.cuda().reshape((B,) + plan.shape)).cpu().numpy()
    ref = oracle.adjoint(sc, x.numpy()).reshape(y.shape)
    assert_parity(y, ref, TOL_F32, what=f"adjoint case {case}, {B} frames")
    plan.close()


@pytest.mark.parametrize("rows", [7, 16, 64, 0, 100000])
@pytest.mark.parametrize("case", [0, 3])
def test_adjoint_row_bands(das, oracle, case, rows):
    """Bands of 7, 16, 64 (and the automatic height) sample rows per CTA, and
    one band holding all K rows: every band boundary splits the interpolation
    taps of some terms between two CTAs, which must still add up exactly."""
    sc = ragged_scene(*RAGGED[case])
    B = 2
    x = image_like(sc, B, seed=80 + case)
    plan = das.Plan.from_scene(sc, max_batch=B)
    plan.set_tuning(adjoint_rows=rows)
    y = plan.adjoint(x.cuda().reshape((B,) + plan.shape)).cpu().numpy()
    plan.close()
    assert_parity(y, oracle.adjoint(sc, x.numpy()).reshape(y.shape), TOL_F32, what=f"adjoint, {rows} rows per band")


@pytest.mark.parametrize("B", [9, 45])
def test_adjoint_and_grad_c_large_batches(das, oracle, B):
    """Batches that span several frame chunks of the adjoint and of the
    derivative kernel (ragged last chunk)."""
    sc = ragged_scene(*RAGGED[0])
    x = image_like(sc, B, seed=50 + B)
    y = S.random_channels(sc, B, seed=60 + B)
    plan = das.Plan.from_scene(sc, max_batch=B)
    ya = plan.adjoint(x.cuda().reshape((B,) + plan.shape)).cpu().numpy()
    assert_parity(ya, oracle.adjoint(sc, x.numpy()).reshape(ya.shape), TOL_F32, what=f"adjoint {B} frames")
    got = float(plan.grad_c(y.cuda(), x.cuda().reshape((B,) + plan.shape)))
    ref = oracle.grad_c(sc, y.numpy(), x.numpy())
    assert abs(got - ref) <= 1e-4 * abs(ref)
    plan.close()


@pytest.mark.parametrize("iq", [False, True])
def test_adjoint_small_and_dot_product(das, oracle, iq):
    """Full-size small scene, and <A y, x> = <y, A^H x> with both maps on the GPU."""
    sc = S.scene_small_iq() if iq else S.scene_small()
    B = 2
    x = image_like(sc, B, seed=3)
    y = S.random_channels(sc, B, seed=4)
    plan = das.Plan.from_scene(sc, max_batch=B)
    ya = plan.adjoint(x.cuda().reshape((B,) + plan.shape))
    ref = oracle.adjoint(sc, x.numpy()).reshape(ya.shape)
    assert_parity(ya.cpu().numpy(), ref, TOL_F32, what="adjoint small scene")
    Ay = plan.forward(y.cuda()).reshape(B, -1)
    lhs = torch.vdot(Ay.reshape(-1).to(torch.complex128), x.cuda().reshape(-1).to(torch.complex128))
    rhs = torch.vdot(y.cuda().reshape(-1).to(torch.complex128), ya.reshape(-1).to(torch.complex128))
    scale = float(torch.linalg.norm(Ay.double() if not iq else Ay.to(torch.complex128)) *
                  torch.linalg.norm(x.double() if not iq else x.to(torch.complex128)))
    assert abs(complex(lhs) - complex(rhs)) <= 1e-5 * scale
    plan.close()


def test_adjoint_diff_scale_sampled_rows(das, oracle):
    """96^3 voxels x 1024 elements x 8 transmits, K = 1536: sampled channel rows."""
    sc = S.scene_diff()
    x = image_like(sc, 1, seed=7)
    plan = das.Plan.from_scene(sc, max_batch=1)
    y = plan.adjoint(x.cuda().reshape((1,) + plan.shape)).reshape(1, sc.Q * sc.M, sc.K)
    rows = np.array([0, 517, 1023 + 3 * 1024, 7 * 1024 + 500, 4 * 1024 + 255])
    ref = oracle.adjoint(sc, x.numpy(), rows=rows)
    got = y[:, torch.as_tensor(rows, device="cuda")].cpu().numpy()
    assert_parity(got, ref, TOL_F32, what="adjoint sampled rows")
    plan.close()


@pytest.mark.parametrize("case", [0, 2, 3])
@pytest.mark.parametrize("B", [1, 3])
def test_grad_c_matches_oracle(das, oracle, case, B):
    sc = ragged_scene(*RAGGED[case])
    y = S.random_channels(sc, B, seed=30 + case)
    g = image_like(sc, B, seed=40 + case)
    plan = das.Plan.from_scene(sc, max_batch=B)
    got = float(plan.grad_c(y.cuda(), g.cuda().reshape((B,) + plan.shape)))
    ref = oracle.grad_c(sc, y.numpy(), g.numpy())
    assert abs(got - ref) <= 1e-4 * abs(ref)
    plan.close()


def test_grad_c_rf(das, oracle):
    """RF data sampled at 16 samples per period.  The derivative of the
    interpolant jumps at integer delays, where the float32 kernel and the
    float64 oracle may pick neighbouring cells; fine sampling keeps those
    jumps small next to the 1e-4 bar."""
    sc = S.scene_small().with_(fs=120e6, K=2048)
    y = S.frames(sc, 1, seed=1, n_speckle=2000, points=S.SMALL_POINTS)
    g = image_like(sc, 1, seed=5)
    plan = das.Plan.from_scene(sc)
    got = float(plan.grad_c(y.cuda(), g.cuda().reshape((1,) + plan.shape)))
    ref = oracle.grad_c(sc, y.numpy(), g.numpy())
    assert abs(got - ref) <= 1e-4 * abs(ref)
    plan.close()


@pytest.mark.parametrize("c_true,offset", [(1480.0, 40.0), (1540.0, -40.0), (1600.0, -40.0)])
def test_autograd_sound_speed_sweep(das, oracle, c_true, offset):
    """Differentiation form: data simulated at c_true, beamformed at
    c_true + offset; dL/dc of L = -sum|x|^4 / (sum|x|^2)^2 through
    torch.autograd against the oracle's derivative, and its sign."""
    sc = S.scene_small_iq().with_(tx_kind=np.array([0, 0], np.int32),
                                  tx_vec=np.array([[-1.5e-3, 0, -10e-3], [1.5e-3, 0, -10e-3]]))
    y = S.frames(sc, 1, seed=5, n_speckle=400, points=S.SMALL_POINTS, c=c_true)
    c_bf = c_true + offset
    plan = das.Plan.from_scene(sc, c=c_bf)
    c = torch.tensor(c_bf, dtype=torch.float64, requires_grad=True)
    yc = y.cuda().requires_grad_(True)
    img = das.das(yc, c, plan)
    loss = -(img.abs() ** 4).sum() / (img.abs() ** 2).sum() ** 2
    loss.backward()
    x_ref = oracle.forward(sc.with_(c=c_bf), y.numpy())
    _, gref = oracle.loss_and_cotangent(x_ref)
    ref = oracle.grad_c(sc.with_(c=c_bf), y.numpy(), gref)
    assert abs(float(c.grad) - ref) <= 1e-3 * abs(ref)
    assert np.sign(float(c.grad)) == np.sign(offset)
    # the y-gradient is the adjoint of the image cotangent
    gx = torch.as_tensor(gref.astype(np.complex64)).cuda().reshape((1,) + plan.shape)
    ya = plan.adjoint(gx)
    assert rel_l2(yc.grad.cpu().numpy(), ya.cpu().numpy()) <= 1e-3
    plan.close()
