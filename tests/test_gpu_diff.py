"""Differentiation workload at full size: 96^3 voxels x 1024 elements x 8
transmits, IQ, 1536 samples.  Data simulated at c_true, beamformed at
c_true +- 40 m/s.  dL/dc of L = -sum|x|^4 / (sum|x|^2)^2 through
torch.autograd is checked against central differences of the GPU forward
pass (h = 0.05 m/s), against the FP64 oracle's derivative on a voxel subset,
and for its sign; the adjoint passes the dot-product test."""
import numpy as np
import pytest
import torch

from paper_2606_13259_gb300 import synth as S
from test_gpu_forward import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def das():
    import __graft_entry__ as G

    G.build()
    import paper_2606_13259_gb300 as P

    torch.cuda.set_device(0)
    return P


def loss_of(img):
    a2 = img.abs().double() ** 2
    return -(a2 * a2).sum() / a2.sum() ** 2


@pytest.mark.parametrize("c_true", [1480.0, 1540.0, 1600.0])
@pytest.mark.parametrize("offset", [-40.0, 40.0])
def test_sound_speed_gradient_full_size(das, oracle, c_true, offset):
    c_bf = c_true + offset
    sc = S.scene_diff(c=c_bf)
    y = S.frames(sc, 1, seed=5, n_speckle=20000, points=S.paper_points(sc), c=c_true, device="cuda")
    plan = das.Plan.from_scene(sc)
    c = torch.tensor(c_bf, dtype=torch.float64, requires_grad=True)
    img = das.das(y, c, plan)
    loss = loss_of(img)
    loss.backward()
    grad = float(c.grad)
    h = 0.05
    with torch.no_grad():
        plan.set_c(c_bf + h)
        lp = float(loss_of(plan.forward(y)))
        plan.set_c(c_bf - h)
        lm = float(loss_of(plan.forward(y)))
        plan.set_c(c_bf)
    fd = (lp - lm) / (2 * h)
    print(f"c_true {c_true} c_bf {c_bf}: dL/dc {grad:.6e} fd {fd:.6e}")
    assert abs(grad - fd) <= 5e-3 * abs(fd)
    assert np.sign(grad) == np.sign(offset)
    # the derivative restricted to a voxel subset against the oracle
    x = img.detach().reshape(1, -1)
    a2 = x.abs().double() ** 2
    s2, s4 = a2.sum(), (a2 * a2).sum()
    g = (2.0 * (-2.0 * x.to(torch.complex128) * (a2 * s2 - s4) / s2 ** 3)).to(torch.complex64)
    rng = np.random.default_rng(int(c_true))
    vox = np.sort(rng.choice(sc.N, 160, replace=False))
    mask = torch.zeros(sc.N, dtype=torch.bool, device="cuda")
    mask[torch.as_tensor(vox, device="cuda")] = True
    g_sub = torch.where(mask, g[0], torch.zeros_like(g[0])).reshape((1,) + plan.shape).contiguous()
    got = float(plan.grad_c(y, g_sub))
    ref = oracle.grad_c(sc, y.cpu().numpy(), g[:, torch.as_tensor(vox, device="cuda")].cpu().numpy(), voxels=vox)
    assert abs(got - ref) <= 1e-3 * abs(ref)
    plan.check()
    plan.close()


def test_adjoint_dot_product_full_size(das):
    sc = S.scene_diff()
    y = S.random_channels(sc, 1, seed=11).cuda()
    x = S.random_image(sc, 1, seed=12).cuda()
    plan = das.Plan.from_scene(sc)
    Ay = plan.forward(y).reshape(-1).to(torch.complex128)
    AHx = plan.adjoint(x.reshape((1,) + plan.shape)).reshape(-1).to(torch.complex128)
    lhs = torch.vdot(Ay, x.reshape(-1).to(torch.complex128))
    rhs = torch.vdot(y.reshape(-1).to(torch.complex128), AHx)
    scale = float(torch.linalg.norm(Ay) * torch.linalg.norm(x.to(torch.complex128)))
    print(f"<Ay,x> {complex(lhs):.6e} <y,A^H x> {complex(rhs):.6e}")
    assert abs(complex(lhs) - complex(rhs)) <= 1e-5 * scale
    plan.close()
