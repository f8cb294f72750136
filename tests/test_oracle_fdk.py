"""Pins of the oracle's FDK pieces (Sec. 2.1, direct methods): the Ram-Lak
frequency response, the cosine pre-weight, the distance-weighted
backprojection of a constant and the reconstruction of a uniform ball from
its analytic projections."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def _row_geo(nu, du=1.0, n_angles=1, nv=1):
    return inputs.circular_geometry((4, 4, 4), (1.0,) * 3, (nu, nv), (du, 1.0), n_angles, 1000.0, 1000.0)


def test_ramlak_passes_ramp_response():
    """The sampled band-limited ramp kernel has DTFT |w| below Nyquist, so a
    cosine of frequency w0 (cycles/mm at the isocentre) comes back scaled by
    w0, up to the truncation of the kernel at the row ends (~1/(pi^2 tau K))."""
    nu = 2048
    g = _row_geo(nu, du=1.0)
    tau = 1.0  # du * DSO / DSD
    iu = np.arange(nu)
    for period in (8.0, 16.0, 5.0):
        w0 = 1.0 / (period * tau)
        row = np.cos(2 * math.pi * w0 * tau * (iu - nu / 2))
        # the cosine pre-weight is 1 up to 2e-7 on the central row near the
        # middle; undo it exactly to isolate the filter
        f = oracle.frames(g)
        P = oracle.pixel_centres(g, 0)[0]
        dirs = P - f["S"][0]
        wcos = np.abs(dirs @ f["n"][0]) / np.linalg.norm(dirs, axis=1)
        out = oracle.fdk_filter(g, (row / wcos)[None, None, :])[0, 0]
        mid = slice(nu // 2 - 64, nu // 2 + 64)
        bound = 2.0 / (math.pi ** 2 * (nu / 2 - 64))
        np.testing.assert_allclose(out[mid], w0 * row[mid], atol=bound)


def test_ramlak_dc_gain_vanishes():
    nu = 4096
    g = _row_geo(nu, du=0.5)
    tau = 0.5
    f = oracle.frames(g)
    P = oracle.pixel_centres(g, 0)[0]
    dirs = P - f["S"][0]
    wcos = np.abs(dirs @ f["n"][0]) / np.linalg.norm(dirs, axis=1)
    out = oracle.fdk_filter(g, (1.0 / wcos)[None, None, :])[0, 0]
    K = nu // 2 - 8
    # tail of sum_{k odd > K} 2/(k^2 pi^2 tau^2), times tau
    assert abs(out[nu // 2]) < tau * 1.0 / (math.pi ** 2 * tau * tau * K)
    assert abs(out[nu // 2]) < 1e-3 * (tau / (4 * tau * tau))


def test_cosine_preweight_ratio():
    """Impulses at the detector centre region and corner: the filtered outputs
    at the impulse positions differ by the cosine of the corner ray angle."""
    nu, nv = 64, 48
    g = inputs.circular_geometry((4, 4, 4), (1.0,) * 3, (nu, nv), (2.0, 2.5), 1, 700.0, 1100.0)
    p = np.zeros(g.proj_shape)
    p[0, 0, 0] = 1.0
    p[0, nv // 2, nu // 2] = 1.0
    out = oracle.fdk_filter(g, p)[0]
    u0, v0 = (0.5 - nu / 2) * 2.0, (0.5 - nv / 2) * 2.5
    uc, vc = 0.5 * 2.0, 0.5 * 2.5
    w0 = 1100.0 / math.sqrt(1100.0 ** 2 + u0 ** 2 + v0 ** 2)
    wc = 1100.0 / math.sqrt(1100.0 ** 2 + uc ** 2 + vc ** 2)
    assert out[0, 0] / out[nv // 2, nu // 2] == pytest.approx(w0 / wc, rel=1e-12)


def test_fdk_backprojection_of_constant():
    """Unfiltered constant 1 projections backprojected with (DSO/L)^2 and
    angle weight pi/nA: the orbit average of (1 - e cos t)^-2 is
    (1 - e^2)^-3/2 with e = r/DSO, so x = pi (1 - (r/DSO)^2)^-3/2."""
    g = inputs.circular_geometry((9, 9, 5), (10.0, 10.0, 10.0), (300, 40), (1.0, 1.0), 64, 100.0, 160.0)
    x = oracle.backproject(g, np.ones(g.proj_shape), "fdk")
    cx = inputs.voxel_centres_1d(9, 10.0)
    r = np.sqrt(cx[None, :] ** 2 + cx[:, None] ** 2)
    ref = math.pi * (1 - (r / 100.0) ** 2) ** -1.5
    np.testing.assert_allclose(x[2], ref, rtol=1e-9)


def ball_projections(geo, radius, mu, centre=(0.0, 0.0, 0.0)):
    f = oracle.frames(geo)
    out = np.zeros(geo.proj_shape)
    c = np.asarray(centre, float)
    for a in range(geo.nAngles):
        P = oracle.pixel_centres(geo, a)
        S = f["S"][a]
        dh = (P - S) / np.linalg.norm(P - S, axis=-1, keepdims=True)
        w = c - S
        r2 = np.sum(w * w) - np.sum(dh * w, axis=-1) ** 2
        out[a] = mu * 2.0 * np.sqrt(np.maximum(radius * radius - r2, 0.0))
    return out


def test_fdk_reconstructs_uniform_ball():
    """FDK of the analytic projections of a uniform ball (radius 20 mm,
    mu 0.02 /mm) in the 64^3 workload geometry returns mu in the central
    region within 2 %."""
    g = inputs.config_small()
    b = ball_projections(g, 20.0, 0.02)
    x = oracle.fdk(g, b)
    c = inputs.voxel_centres_1d(64, 1.0)
    R = np.sqrt(c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2)
    inner = R < 12.0
    assert np.abs(x[inner] / 0.02 - 1.0).max() < 0.02
    # outside the ball, inside the fully sampled field of view: view-aliasing
    # streaks of 100 views average out to near zero
    r = np.sqrt(c[None, None, :] ** 2 + c[None, :, None] ** 2 + 0 * c[:, None, None])
    Z = np.abs(c[:, None, None] + 0 * c[None, None, :] + 0 * c[None, :, None])
    shell = (R > 24.0) & (r < 30.0) & (Z < 24.0)
    assert abs(x[shell].mean()) < 0.005 * 0.02
    assert np.abs(x[shell]).mean() < 0.03 * 0.02


@pytest.mark.parametrize("which", ["u", "v"])
def test_fdk_backprojection_of_linear_projection(which):
    """Bilinear interpolation reproduces a projection that is linear in the
    pixel index, so one view of p = iu (or iv) backprojects to
    pi * (DSO/L)^2 * fu (or fv) with the perspective position worked out by
    hand for the untilted view at angle 0: L = DSO - x,
    fu = (y DSD / L) / du + nu/2 - 1/2, fv = (z DSD / L) / dv + nv/2 - 1/2."""
    nu, nv = 200, 150
    DSO, DSD, du, dv = 300.0, 500.0, 0.7, 0.9
    g = inputs.circular_geometry((7, 6, 5), (3.0, 2.5, 4.0), (nu, nv), (du, dv), 1, DSO, DSD)
    iu, iv = np.meshgrid(np.arange(nu), np.arange(nv))
    p = (iu if which == "u" else iv).astype(float)[None]
    x = oracle.backproject(g, p, "fdk")
    cx, cy, cz = (inputs.voxel_centres_1d(n, d) for n, d in zip(g.nVoxel, g.dVoxel))
    X, Y, Z = cx[None, None, :], cy[None, :, None], cz[:, None, None]
    L = DSO - X
    if which == "u":
        f = (Y * DSD / L) / du + nu / 2 - 0.5
    else:
        f = (Z * DSD / L) / dv + nv / 2 - 0.5
    ref = np.broadcast_to(math.pi * (DSO / L) ** 2 * f, x.shape)
    np.testing.assert_allclose(x, ref, rtol=1e-11)
