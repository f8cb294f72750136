"""GPU parity of the TV kernels and ASD-POCS (Sec. 2.1 POCS methods; AwTV
of the algorithm features in Sec. 2.2) against the FP64 oracle.

Tolerances: the gradient and the descent steps are FP32 evaluations of a
smooth closed form (relative L2 <= 1e-5); ASD-POCS after its iterations
<= 1e-4, the bar of the iterative solvers."""
import math

import numpy as np
import pytest

import oracle
from conftest import max_rel, rel_l2
from oracle import tv as otv
from paper_2412_10129_gb300 import inputs, tg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_10129_gb300 import build
    build.build()
    tg.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape", [(23, 29, 37), (1, 1, 40), (5, 1, 1), (64, 64, 64), (70, 9, 33)])
@pytest.mark.parametrize("delta", [math.inf, 0.02])
def test_tv_gradient_matches_oracle(shape, delta):
    g = inputs.circular_geometry(shape[::-1], (1.0,) * 3, (8, 8), (1.0, 1.0), 1, 500.0, 800.0)
    x = inputs.ellipsoid_phantom(g, 6, seed=51) + 0.003 * inputs.random_volume(g, seed=52)
    got = host(tg.tv_gradient(dev(x), delta=delta, eps=1e-8))
    ref = otv.awtv_gradient(x.astype(np.float32), delta, 1e-8)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    assert max_rel(got, ref) <= 1e-4, max_rel(got, ref)


@pytest.mark.parametrize("delta", [math.inf, 0.02])
def test_tv_descent_matches_oracle(delta):
    g = inputs.circular_geometry((30, 26, 20), (1.0,) * 3, (8, 8), (1.0, 1.0), 1, 500.0, 800.0)
    x = inputs.ellipsoid_phantom(g, 6, seed=53) + 0.005 * inputs.random_volume(g, seed=54)
    t = dev(x)
    tg.tv_descent(t, 7, 0.05, delta=delta)
    ref = otv.tv_descent(x.astype(np.float32), 7, 0.05, delta)
    assert rel_l2(host(t), ref) <= 1e-5, rel_l2(host(t), ref)


@pytest.mark.parametrize("blocksize,delta", [(10, math.inf), (1, math.inf), (20, 0.01)])
def test_asd_pocs_matches_oracle(blocksize, delta):
    g = inputs.circular_geometry((32, 32, 16), (1.0,) * 3, (48, 24), (1.0, 1.0), 40, 300.0, 450.0)
    xt = inputs.ellipsoid_phantom(g, 5, seed=55)
    b = oracle.forward(g, xt)
    b = (b + np.random.default_rng(56).normal(0, 0.01 * b.max(), b.shape)).astype(np.float32)
    x, h = tg.asd_pocs(g, dev(b), 4, blocksize=blocksize, delta=delta, resid=True)
    xr, hr = otv.asd_pocs(g, b, 4, blocksize=blocksize, delta=delta)
    assert rel_l2(host(x), xr) <= 1e-4, rel_l2(host(x), xr)
    np.testing.assert_allclose(h, hr, rtol=1e-4)
