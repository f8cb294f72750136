"""Pins of the oracle's interpolated projector and its transpose.

The interpolated projector reads Eq. 1 as b_i = delta * sum_k f(S + k delta d_i)
over the samples k >= 0 that lie in the closed volume box and on the segment
from the source to the pixel, with f the trilinear interpolant of the voxel
values (zero outside the grid).  The pins below do not reuse the oracle's
arithmetic: a brute-force evaluation of that definition through the
tent-function basis, the line integral of a Gaussian blob (closed form), a
translation identity, and the adjoint identity for the transpose."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def brute_force_interp(geo, vol, a, iu, iv):
    """f(p) = sum_j x_j prod_axes max(0, 1 - |p_axis/d - (j+0.5-n/2)|) over
    ALL voxels; every k from 0 to |P-S|/delta is tested for box membership."""
    f = oracle.frames(geo)
    S = f["S"][a]
    P = oracle.pixel_centres(geo, a)[iv, iu]
    L = np.linalg.norm(P - S)
    dh = (P - S) / L
    delta = geo.accuracy * min(geo.dVoxel)
    n = np.asarray(geo.nVoxel)
    d = np.asarray(geo.dVoxel)
    h = 0.5 * n * d
    cs = [((np.arange(n[i]) + 0.5) - 0.5 * n[i]) * d[i] for i in range(3)]
    total = 0.0
    for k in range(int(math.floor(L / delta)) + 1):
        p = S + k * delta * dh
        if np.any(p < -h) or np.any(p > h):
            continue
        tx = np.maximum(0.0, 1.0 - np.abs(p[0] - cs[0]) / d[0])
        ty = np.maximum(0.0, 1.0 - np.abs(p[1] - cs[1]) / d[1])
        tz = np.maximum(0.0, 1.0 - np.abs(p[2] - cs[2]) / d[2])
        total += np.einsum("zyx,z,y,x->", vol, tz, ty, tx)
    return delta * total


@pytest.mark.parametrize("seed", [0, 1])
def test_interp_matches_brute_force_definition(seed):
    g = inputs.random_geometry((5, 4, 3), (1.0, 1.3, 0.8), (7, 6), (1.1, 0.9), 3, seed=seed,
                               DSO=40.0, DSD=70.0)
    g.accuracy = 0.37
    vol = np.random.default_rng(seed).random(g.vol_shape)
    proj = oracle.forward(g, vol, "interp")
    for a in range(g.nAngles):
        for iv in range(g.nDetector[1]):
            for iu in range(g.nDetector[0]):
                ref = brute_force_interp(g, vol, a, iu, iv)
                assert proj[a, iv, iu] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_interp_gaussian_line_integrals():
    """A Gaussian blob of width s has line integral s sqrt(2 pi) exp(-r^2/(2 s^2))
    along a line at distance r from its centre; trilinear sampling of a blob of
    several voxels converges to it at second order in the voxel size."""
    g = inputs.circular_geometry((48, 48, 48), (1.0,) * 3, (40, 40), (1.0, 1.0), 3, 1000.0, 1536.0)
    g.accuracy = 0.25
    s = 6.0
    m = np.array([2.0, -3.0, 1.5])
    c = [inputs.voxel_centres_1d(n, d) for n, d in zip(g.nVoxel, g.dVoxel)]
    X, Y, Z = c[0][None, None, :], c[1][None, :, None], c[2][:, None, None]
    vol = np.exp(-((X - m[0]) ** 2 + (Y - m[1]) ** 2 + (Z - m[2]) ** 2) / (2 * s * s))
    proj = oracle.forward(g, vol, "interp")
    f = oracle.frames(g)
    for a in range(g.nAngles):
        P = oracle.pixel_centres(g, a)
        S = f["S"][a]
        dh = (P - S) / np.linalg.norm(P - S, axis=-1, keepdims=True)
        w = m - S
        r2 = np.sum(w * w) - np.sum(dh * w, axis=-1) ** 2
        ref = s * math.sqrt(2 * math.pi) * np.exp(-r2 / (2 * s * s))
        central = ref > 0.3 * ref.max()
        err = np.abs(proj[a] - ref)[central] / ref[central]
        # Linear interpolation of f between samples h apart is biased by
        # f'' d (h - d) / 2 at offset d, at most f'' h^2 / 8.  Rays running
        # almost along x keep their y and z offsets, so the worst central-ray
        # bias is 2 * (h^2/8) / s^2 = h^2 / (4 s^2) relative (0.69 % here);
        # allow 30 % for higher-order terms.
        assert err.max() < 1.3 * 1.0 / (4 * s * s)


def test_interp_translation_identity():
    """Moving the volume by one voxel along x (offOrigin) and moving its
    content by one index the other way leaves every projection unchanged,
    because the sample lattice is fixed to the source."""
    g = inputs.circular_geometry((12, 10, 8), (1.0, 0.9, 1.1), (20, 14), (1.3, 1.3), 5, 200.0, 350.0)
    vol = np.zeros(g.vol_shape)
    vol[2:-2, 2:-2, 2:-2] = np.random.default_rng(3).random((4, 6, 8))
    p0 = oracle.forward(g, vol, "interp")
    g2 = inputs.circular_geometry((12, 10, 8), (1.0, 0.9, 1.1), (20, 14), (1.3, 1.3), 5, 200.0, 350.0)
    g2.offOrigin = np.tile([1.0, 0.0, 0.0], (5, 1))
    vol2 = np.zeros_like(vol)
    vol2[:, :, :-1] = vol[:, :, 1:]
    p1 = oracle.forward(g2, vol2, "interp")
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-12 * p0.max())


def test_interp_zero_and_miss():
    g = inputs.circular_geometry((6, 6, 6), (1.0,) * 3, (8, 8), (1.0, 1.0), 2, 100.0, 150.0)
    assert np.all(oracle.forward(g, np.zeros(g.vol_shape), "interp") == 0)
    # detector far off to the side: no ray meets the volume
    g.offDetector = np.array([[500.0, 0.0], [500.0, 0.0]])
    assert np.all(oracle.forward(g, np.ones(g.vol_shape), "interp") == 0)


@pytest.mark.parametrize("kind", ["circular", "random"])
def test_matched_adjoint_identity(kind):
    if kind == "circular":
        g = inputs.circular_geometry((11, 9, 7), (1.0, 1.1, 0.9), (15, 12), (1.2, 1.0), 6, 120.0, 200.0)
    else:
        g = inputs.random_geometry((9, 10, 8), (1.0, 1.0, 1.2), (14, 13), (1.1, 1.0), 5, seed=7,
                                   DSO=100.0, DSD=170.0)
    rng = np.random.default_rng(11)
    x = rng.random(g.vol_shape)
    y = rng.random(g.proj_shape)
    lhs = float(np.sum(oracle.forward(g, x, "interp") * y))
    rhs = float(np.sum(x * oracle.backproject(g, y, "matched")))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_matched_gather_form_equals_scatter():
    g = inputs.random_geometry((9, 8, 7), (1.0, 1.2, 0.9), (16, 14), (1.0, 1.1), 4, seed=5,
                               DSO=90.0, DSD=160.0)
    y = np.random.default_rng(2).random(g.proj_shape)
    full = oracle.backproject(g, y, "matched")
    vox = np.array([[0, 0, 0], [8, 7, 6], [4, 3, 2], [1, 7, 3], [8, 0, 5], [5, 5, 0]])
    got = oracle.backproject_voxels(g, y, vox, "matched")
    ref = full[vox[:, 2], vox[:, 1], vox[:, 0]]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_rays_subset_equals_full():
    g = inputs.random_geometry((9, 8, 7), (1.0,) * 3, (10, 9), (1.3, 1.2), 3, seed=9, DSO=80.0, DSD=150.0)
    vol = np.random.default_rng(0).random(g.vol_shape)
    for method in ("interp", "siddon"):
        full = oracle.forward(g, vol, method)
        rays = np.array([[0, 0, 0], [2, 8, 9], [1, 4, 5], [2, 3, 1]])
        got = oracle.forward_rays(g, vol, rays, method)
        np.testing.assert_array_equal(got, full[rays[:, 0], rays[:, 1], rays[:, 2]])
