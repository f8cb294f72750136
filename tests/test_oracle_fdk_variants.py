"""Pins of the oracle's FDK variants (Sec. 2.1, direct methods: filter
types, Parker and Wang weights): the frequency-domain filter against the
spatial Ram-Lak filter and the classical Shepp-Logan kernel, the windows'
responses to cosines, the redundancy of Parker and Wang weights on rays
whose conjugates are found by geometry, and short-scan / displaced-detector
reconstructions of uniform balls."""
import math

import numpy as np
import pytest

import oracle
from oracle import fdk_variants as ofdk
from paper_2412_10129_gb300 import inputs
from test_oracle_fdk import ball_projections


def test_frequency_filter_equals_spatial_ramlak():
    """With the flat window the frequency-domain path is the linear
    convolution with the Ram-Lak kernel, i.e. the C oracle's spatial filter,
    for arbitrary per-angle geometry (tilts, offsets, per-angle DSO/DSD)."""
    g = inputs.random_geometry((8, 8, 8), (1.0,) * 3, (37, 11), (0.9, 1.1), 5, seed=3)
    p = np.random.default_rng(4).standard_normal(g.proj_shape)
    a = ofdk.fdk_filter(g, p, "ram-lak")
    b = oracle.fdk_filter(g, p)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


# Window values at f = 1/16, 1/8 and 1/4 cycles per sample (closed forms):
#   shepp-logan sin(pi f)/(pi f), cosine cos(pi f), hamming 0.54 + 0.46 cos(2 pi f),
#   hann 0.5 + 0.5 cos(2 pi f).
WINDOW_VALUES = {
    "ram-lak": (1.0, 1.0, 1.0),
    "shepp-logan": (0.99359432, 0.97449536, 0.90031632),
    "cosine": (0.98078528, 0.92387953, 0.70710678),
    "hamming": (0.96498904, 0.86526912, 0.54),
    "hann": (0.96193977, 0.85355339, 0.5),
}


@pytest.mark.parametrize("name", ofdk.WINDOWS)
def test_window_response_to_cosines(name):
    """A cosine of f0 cycles per sample comes back scaled by f0 W(f0) / tau
    in the middle of a long row (up to the kernel's truncation at the row
    ends, ~2 / (pi^2 distance))."""
    nu, tau = 2048, 0.7
    iu = np.arange(nu)
    mid = slice(nu // 2 - 64, nu // 2 + 64)
    bound = 2.0 / (math.pi ** 2 * (nu / 2 - 64)) / tau
    for f0, wv in zip((1 / 16, 1 / 8, 1 / 4), WINDOW_VALUES[name]):
        row = np.cos(2 * math.pi * f0 * (iu - nu / 2) + 0.3)
        out = ofdk.filter_rows(row[None], np.array([tau]), name)[0]
        np.testing.assert_allclose(out[mid], f0 * wv / tau * row[mid], atol=bound)


def test_nyquist_row():
    """The alternating row (f = 1/2): Ram-Lak passes 1/2, Hamming 0.08 * 1/2,
    Hann and cosine remove it, Shepp-Logan passes (2/pi) * 1/2."""
    nu = 2048
    row = (-1.0) ** np.arange(nu)
    mid = slice(nu // 2 - 64, nu // 2 + 64)
    bound = 2.0 / (math.pi ** 2 * (nu / 2 - 64))
    for name, gain in (("ram-lak", 0.5), ("hamming", 0.04), ("hann", 0.0), ("cosine", 0.0),
                       ("shepp-logan", 1.0 / math.pi)):
        out = ofdk.filter_rows(row[None], np.array([1.0]), name)[0]
        np.testing.assert_allclose(out[mid], gain * row[mid], atol=bound)


def test_shepp_logan_matches_classical_kernel():
    """The Shepp-Logan window on the Ram-Lak response against the classical
    spatial kernel h[n] = -2 / (pi^2 tau^2 (4 n^2 - 1)) (times tau), whose
    response is exactly |f| sinc(f): the two differ only by the Ram-Lak
    kernel's truncation at N/2 (response error < 1 / (pi^2 N/2))."""
    nu, tau = 300, 1.3
    rng = np.random.default_rng(8)
    rows = rng.standard_normal((6, nu))
    got = ofdk.filter_rows(rows, np.full(6, tau), "shepp-logan")
    n = np.arange(-(nu - 1), nu)
    h = -2.0 / (math.pi ** 2 * (4.0 * n * n - 1.0)) / tau
    ref = np.stack([np.convolve(r, h)[nu - 1:2 * nu - 1] for r in rows])
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    N = ofdk.fft_length(nu)
    assert err < 4.0 / (math.pi ** 2 * N / 2)
    # the cosine window would be far off
    other = ofdk.filter_rows(rows, np.full(6, tau), "cosine")
    assert np.linalg.norm(other - ref) / np.linalg.norm(ref) > 0.05


def _fan_row_geometry(angles, nu=16, du=6.0, DSO=1000.0, DSD=1536.0):
    g = inputs.circular_geometry((4, 4, 4), (1.0,) * 3, (nu, 1), (du, 1.0), len(angles), DSO, DSD)
    g.angles[:, 0] = angles
    return g


def _conjugate(S, P, DSO):
    """The other source position on the orbit circle along the line S -> P,
    as an orbit angle."""
    d = P - S
    d2 = d[:2]
    t = -2.0 * (S[:2] @ d2) / (d2 @ d2)
    Q = S + t * d
    return math.atan2(Q[1], Q[0]) % (2 * math.pi)


def test_parker_weights_of_conjugate_rays_sum_to_one():
    """For rays in the first transition region, the conjugate ray (the same
    line seen from the other end, found by intersecting the line with the
    source orbit) lies in the last one, at the mirrored pixel; the two
    Parker weights sum to 1.  Rays of the middle region weigh 1, the end
    projections 0."""
    nu, DSO, Delta = 16, 1000.0, math.radians(10.0)
    bmax = math.pi + 2 * Delta
    for iu in (0, 3, 7, 8, 12, 15):
        probe = _fan_row_geometry([0.0, 0.2, bmax])
        f = oracle.frames(probe)
        P = oracle.pixel_centres(probe, 1)[0, iu]
        b2 = _conjugate(f["S"][1], P, DSO)
        g = _fan_row_geometry([0.0, 0.2, b2, bmax])
        Pc = oracle.pixel_centres(g, 2)[0]
        fc = oracle.frames(g)
        # the line crosses the detector of angle b2 at the mirrored pixel
        d = P - fc["S"][2]
        assert np.linalg.norm(np.cross(d, Pc[nu - 1 - iu] - fc["S"][2])) < 1e-9 * np.linalg.norm(d) ** 2
        w = ofdk.pre_weights(g, parker=True) / ofdk.pre_weights(g)
        assert 0.0 < w[1, 0, iu] < 1.0
        assert w[1, 0, iu] + w[2, 0, nu - 1 - iu] == pytest.approx(1.0, abs=1e-12)
        np.testing.assert_allclose(w[0], 0.0, atol=1e-15)
        np.testing.assert_allclose(w[3], 0.0, atol=1e-12)
    mid = _fan_row_geometry([0.0, 1.2, 2.0, bmax])
    w = ofdk.pre_weights(mid, parker=True) / ofdk.pre_weights(mid)
    np.testing.assert_allclose(w[1:3], 1.0)
    # the central ray (odd detector: gamma = 0) is half weighted in the
    # middle of both transitions, which span 2 Delta each
    half = _fan_row_geometry([0.0, Delta, math.pi + Delta, bmax], nu=17)
    w = ofdk.pre_weights(half, parker=True) / ofdk.pre_weights(half)
    assert w[1, 0, 8] == pytest.approx(0.5, abs=1e-12)
    assert w[2, 0, 8] == pytest.approx(0.5, abs=1e-12)


def _short_scan(n_angles=120, arc_deg=200.0):
    g = inputs.config_small()
    arc = math.radians(arc_deg)
    return inputs.circular_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, n_angles,
                                    1000.0, 1536.0, arc=arc * n_angles / (n_angles - 1))


@pytest.mark.parametrize("centre,radius", [((0.0, 0.0, 0.0), 20.0), ((12.0, -9.0, 0.0), 12.0)])
def test_parker_short_scan_reconstructs_ball(centre, radius):
    """A 200-degree scan of a uniform ball (mu 0.02): Parker-weighted FDK
    returns mu inside the ball within 0.5 %.  Without the redundancy weights
    (the full-orbit angle weight pi / nAngles, whose total is the same) the
    error is ten times larger."""
    g = _short_scan()
    b = ball_projections(g, radius, 0.02, centre)
    x = ofdk.fdk(g, b, parker=True)
    c = inputs.voxel_centres_1d(64, 1.0)
    X, Y, Z = c[None, None, :], c[None, :, None], c[:, None, None]
    R = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    inner = R < 0.6 * radius
    assert np.abs(x[inner] / 0.02 - 1.0).max() < 0.005
    plain = ofdk.fdk(g, b)
    assert np.abs(plain[inner] / 0.02 - 1.0).max() > 0.01


def _offset_geometry(n_angles=100, shift_px=40):
    g = inputs.config_small()
    g = inputs.circular_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, n_angles, 1000.0, 1536.0)
    g.offDetector[:, 0] = shift_px * g.dDetector[0]
    return g


def test_wang_weights_of_conjugate_pixels_sum_to_two():
    """Displaced detector: u0 is the half-width seen from both sides; mirrored
    pixels about the central ray (conjugate rays of a full orbit) weigh 2 in
    total, pixels beyond u0 on the long side weigh 2."""
    g = _offset_geometry(4, shift_px=40)
    w = ofdk.pre_weights(g, wang=True) / ofdk.pre_weights(g)
    nu, du = 128, 0.8
    # pixel centres at u = (iu + 0.5 - nu/2) du + 40 du; the central ray is
    # at pixel coordinate 23.5, the short side spans 24 pixels
    u = (np.arange(nu) + 0.5 - nu / 2) * du + 40 * du
    assert ofdk.wang_overlap(g, 0) == pytest.approx((24 * du, 1.0))
    for iu in range(0, 24):
        j = int(round((-u[iu] - u[0]) / du))
        assert u[j] == pytest.approx(-u[iu])
        np.testing.assert_allclose(w[:, :, iu] + w[:, :, j], 2.0, atol=1e-12)
    np.testing.assert_allclose(w[:, :, 48:], 2.0)


@pytest.mark.parametrize("centre,radius,shift", [((0.0, 0.0, 0.0), 20.0, 40), ((10.0, 8.0, 0.0), 14.0, 24)])
def test_wang_offset_detector_reconstructs_ball(centre, radius, shift):
    """The detector shifted by 40 (24) of its 128 pixels sees +-12.5 mm
    (+-20.8 mm) of the isocentre plane from both sides; the balls reach
    beyond that, so their shadows are cut on the short side.  Wang-weighted
    FDK returns mu inside the ball within 1 %; without the weights the
    doubly seen region counts twice (errors of tens of percent)."""
    g = _offset_geometry(100, shift)
    b = ball_projections(g, radius, 0.02, centre)
    x = ofdk.fdk(g, b, wang=True)
    c = inputs.voxel_centres_1d(64, 1.0)
    X, Y, Z = c[None, None, :], c[None, :, None], c[:, None, None]
    R = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    inner = R < 0.6 * radius
    assert np.abs(x[inner] / 0.02 - 1.0).max() < 0.01
    plain = ofdk.fdk(g, b)
    assert np.abs(plain[inner] / 0.02 - 1.0).max() > 0.5


def test_parker_and_wang_preconditions():
    with pytest.raises(ValueError):
        ofdk.parker_scan(inputs.circular_geometry((4, 4, 4), (1.0,) * 3, (8, 8), (1.0, 1.0), 10, 500.0, 800.0,
                                                  arc=math.pi * 0.9))
    g = _offset_geometry(2, shift_px=70)
    with pytest.raises(ValueError):
        ofdk.wang_overlap(g, 0)
