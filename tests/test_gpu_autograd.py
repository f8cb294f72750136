"""The differentiable projector (PyTorch operator wrappers, Sec. 2.8) and the
unrolled gradient scheme of Eq. 4, on the GPU.

Checks: the autograd gradient of ||A x - b||^2 against central finite
differences (step 1e-3, 64 random voxels, loss differences over the affected
rays in FP64; 1e-2 relative for the FP32 path) and against the FP64 oracle
gradient 2 A^T (A x - b) (1e-4 relative L2); a batch of 16 volumes in one
launch; the unrolled scheme with and without per-step checkpointing."""
import numpy as np
import pytest

import oracle
from conftest import rel_l2
from paper_2412_10129_gb300 import inputs, tg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_10129_gb300 import build
    build.build()
    tg.load()


def ag():
    from paper_2412_10129_gb300 import autograd
    return autograd


def test_gradient_matches_central_differences():
    g = inputs.config_autograd()          # 128^3, 180 angles, 192^2 at 1.2 mm
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.random(g.vol_shape).astype(np.float32)).cuda().requires_grad_(True)
    b = torch.from_numpy(rng.random(g.proj_shape).astype(np.float32)).cuda()
    r = ag().project(x, g) - b
    loss = torch.sum(r.double() ** 2)
    loss.backward()
    grad = x.grad.detach()
    h = 1e-3
    flat = rng.choice(int(np.prod(g.vol_shape)), 64, replace=False)
    xd = x.detach()
    fd, an = [], []
    for j in flat:
        e = torch.zeros_like(xd).view(-1)
        e[j] = h
        e = e.view(g.vol_shape)
        pp = tg.forward(g, xd + e, "interp").double()
        pm = tg.forward(g, xd - e, "interp").double()
        bd = b.double()
        m = pp != pm                                  # the rays voxel j touches
        diff = torch.sum((pp[m] - pm[m]) * (pp[m] + pm[m] - 2 * bd[m]))
        fd.append(float(diff) / (2 * h))
        an.append(float(grad.view(-1)[j]))
    fd, an = np.array(fd), np.array(an)
    assert np.abs(fd - an).max() <= 1e-2 * np.abs(an).max()
    assert rel_l2(an, fd) <= 1e-2


def test_gradient_matches_oracle():
    g = inputs.circular_geometry((40, 40, 40), (1.0,) * 3, (64, 56), (1.0, 1.0), 48, 500.0, 800.0)
    rng = np.random.default_rng(1)
    x_np = rng.random(g.vol_shape).astype(np.float32)
    b_np = rng.random(g.proj_shape).astype(np.float32)
    x = torch.from_numpy(x_np).cuda().requires_grad_(True)
    loss = torch.sum((ag().project(x, g) - torch.from_numpy(b_np).cuda()).double() ** 2)
    loss.backward()
    ref = 2.0 * oracle.backproject(g, oracle.forward(g, x_np, "interp") - b_np, "matched")
    assert rel_l2(x.grad.cpu().numpy(), ref) <= 1e-4


def test_backproject_operator_gradient_is_forward():
    g = inputs.circular_geometry((24, 24, 24), (1.0,) * 3, (32, 32), (1.2, 1.2), 20, 300.0, 500.0)
    y = torch.rand(g.proj_shape, device="cuda", requires_grad=True)
    w = torch.rand(g.vol_shape, device="cuda")
    torch.sum(ag().backproject(y, g) * w).backward()
    torch.testing.assert_close(y.grad, tg.forward(g, w, "interp"))


def test_batch_of_16_in_one_launch():
    g = inputs.config_autograd()
    xb = torch.rand((16,) + g.vol_shape, device="cuda")
    n0 = tg.launch_count()
    pb = ag().project(xb, g)
    torch.cuda.synchronize()
    assert tg.launch_count() - n0 == 1          # one projector launch for the batch
    for i in (0, 7, 15):
        torch.testing.assert_close(pb[i], tg.forward(g, xb[i].contiguous(), "interp"), rtol=0, atol=0)
    n0 = tg.launch_count()
    vb = ag().backproject(pb, g)
    torch.cuda.synchronize()
    # max-|y| pre-pass, the rays' set-up table (shared by the batch), one brick
    # launch for the batch, the merge of the bricks' rims
    assert tg.launch_count() - n0 == 4
    for i in (0, 15):
        torch.testing.assert_close(vb[i], tg.backproject(g, pb[i].contiguous(), "matched"), rtol=0, atol=0)


def test_operator_norm_power_iteration():
    g = inputs.circular_geometry((16, 16, 16), (1.0,) * 3, (24, 24), (1.0, 1.0), 12, 200.0, 320.0)
    lam = ag().operator_norm_sq(g, iters=60)
    # dense check on the oracle's matrix
    n = int(np.prod(g.vol_shape))
    rng = np.random.default_rng(2)
    v = rng.random(n)
    for _ in range(60):
        v = v / np.linalg.norm(v)
        w = oracle.backproject(g, oracle.forward(g, v.reshape(g.vol_shape), "interp"), "matched").reshape(-1)
        ref = float(v @ w)
        v = w
    assert lam == pytest.approx(ref, rel=1e-4)


def test_unrolled_gd_checkpointing_and_oracle():
    g = inputs.circular_geometry((24, 24, 24), (1.0,) * 3, (40, 32), (1.0, 1.0), 30, 300.0, 500.0)
    x_true = inputs.ellipsoid_phantom(g, 4, seed=6, semi_axes=(2.0, 6.0))
    b_np = oracle.forward(g, x_true, "siddon").astype(np.float32)
    eta = 1.0 / ag().operator_norm_sq(g)
    x0 = torch.zeros(g.vol_shape, device="cuda")
    outs, grads = [], []
    for ck in (True, False):
        b = torch.from_numpy(b_np).cuda().requires_grad_(True)
        x = ag().unrolled_gd(x0, b, g, steps=10, eta=eta, checkpoint=ck)
        torch.sum(x.double() ** 2).backward()
        outs.append(x.detach())
        grads.append(b.grad.detach())
    torch.testing.assert_close(outs[0], outs[1], rtol=0, atol=0)
    torch.testing.assert_close(grads[0], grads[1], rtol=0, atol=0)
    # the same ten steps in FP64 on the oracle
    xo = np.zeros(g.vol_shape)
    for _ in range(10):
        xo = xo - eta * oracle.backproject(g, oracle.forward(g, xo, "interp") - b_np, "matched")
    assert rel_l2(outs[0].cpu().numpy(), xo) <= 1e-4
