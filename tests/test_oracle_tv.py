"""Pins of the oracle's TV pieces (Sec. 2.1 POCS methods; the AwTV of the
algorithm features in Sec. 2.2): closed-form TV / AwTV of steps and ramps,
the boundary terms of the gradient of a ramp, central finite differences of
the functional (plain TV, and AwTV with the weights frozen), descent, and
ASD-POCS without TV steps = OS-SART with the relaxation schedule."""
import math

import numpy as np
import pytest

import oracle
from oracle import tv
from paper_2412_10129_gb300 import inputs


def test_tv_of_a_step_and_a_ramp():
    """A jump h across one plane of ny*nz voxels: TV = ny nz |h|, AwTV =
    ny nz |h| exp(-h^2 / (2 delta^2)); a ramp of slope c along x over nx
    voxels: TV = (nx - 1) ny nz |c| (eps = 0)."""
    nz, ny, nx, h = 4, 5, 6, 0.7
    x = np.zeros((nz, ny, nx))
    x[:, :, 3:] = h
    assert tv.awtv(x, eps=0.0) == pytest.approx(ny * nz * h, rel=1e-14)
    assert tv.awtv(x, delta=0.5, eps=0.0) == pytest.approx(ny * nz * h * math.exp(-h * h / (2 * 0.25)), rel=1e-14)
    c = -0.3
    ramp = np.broadcast_to(c * np.arange(nx), (nz, ny, nx))
    assert tv.awtv(ramp, eps=0.0) == pytest.approx((nx - 1) * ny * nz * abs(c), rel=1e-14)
    # large delta approaches TV
    assert tv.awtv(x, delta=1e6, eps=0.0) == pytest.approx(tv.awtv(x, eps=0.0), rel=1e-12)


def test_gradient_of_a_ramp_lives_on_the_boundary():
    """For a ramp along x every interior voxel's own term and its neighbour's
    cancel: the gradient is -sign(c) on the first plane, +sign(c) on the
    last, 0 elsewhere (eps -> 0)."""
    nz, ny, nx, c = 3, 4, 7, 0.5
    ramp = np.broadcast_to(c * np.arange(nx), (nz, ny, nx)).copy()
    g = tv.awtv_gradient(ramp, eps=1e-20)
    np.testing.assert_allclose(g[:, :, 0], -1.0, atol=1e-12)
    np.testing.assert_allclose(g[:, :, -1], 1.0, atol=1e-12)
    np.testing.assert_allclose(g[:, :, 1:-1], 0.0, atol=1e-12)


@pytest.mark.parametrize("delta", [math.inf, 0.4])
def test_gradient_matches_finite_differences(delta):
    """Central differences (h = 1e-6) of AwTV with the weights of x frozen."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (5, 6, 7))
    w = tv.weights(tv.differences(x), delta)
    g = tv.awtv_gradient(x, delta, eps=1e-3)
    h = 1e-6
    for idx in [(0, 0, 0), (4, 5, 6), (2, 3, 1), (0, 5, 3), (3, 0, 6), (1, 2, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (tv.awtv(xp, eps=1e-3, w=w) - tv.awtv(xm, eps=1e-3, w=w)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_tv_descent_lowers_tv():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (6, 6, 6))
    y = tv.tv_descent(x, 10, 0.01)
    assert tv.awtv(y) < tv.awtv(x)
    assert np.linalg.norm(y - x) == pytest.approx(0.1, rel=1e-3)


def test_asd_pocs_without_tv_steps_is_os_sart_with_the_relaxation_schedule():
    g = inputs.random_geometry((9, 8, 7), (1.0,) * 3, (13, 11), (1.2, 1.1), 6, seed=41, DSO=200.0, DSD=330.0)
    b = oracle.forward(g, inputs.random_volume(g, seed=42))
    x, hist = tv.asd_pocs(g, b, 3, blocksize=2, tv_steps=0, beta=0.9, beta_red=0.8)
    y = np.zeros(g.vol_shape)
    lam = 0.9
    for _ in range(3):
        y, _ = oracle.ossart(g, b, 1, 2, lam=lam, x0=y)
        lam *= 0.8
    np.testing.assert_allclose(x, y, rtol=1e-13, atol=1e-15)
    assert hist[-1] == pytest.approx(np.linalg.norm(oracle.forward(g, y) - b), rel=1e-12)


def test_asd_pocs_lowers_tv_at_similar_data_fit():
    """On noisy data of a piecewise-constant phantom the TV steps lower the
    image's TV against plain OS-SART for the same iterations, keeping the
    data residual within 20 %."""
    g = inputs.circular_geometry((24, 24, 12), (1.0,) * 3, (40, 20), (1.0, 1.0), 30, 300.0, 450.0)
    xt = inputs.ellipsoid_phantom(g, 5, seed=43)
    b = oracle.forward(g, xt)
    b = b + np.random.default_rng(44).normal(0, 0.02 * b.max(), b.shape)
    x, hist = tv.asd_pocs(g, b, 5, blocksize=10)
    y, hy = oracle.ossart(g, b, 5, 10)
    assert tv.awtv(x) < 0.8 * tv.awtv(y)
    assert hist[-1] < 1.2 * hy[-1]
