"""Pins of the oracle's parallel-beam mode (the synchrotron shapes of Sec. 3;
every ray runs along the central direction D - S from S + (P - D) to its
pixel centre P): brute-force tent-basis evaluation of the interpolated
projector, Gaussian line integrals in closed form, Siddon line integrals as
plain column sums at angle 0, the Siddon projector as the limit of the cone
beam with a distant source, adjoint identities, the gather form of the
transpose, and parallel FBP of a uniform ball."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def _par(nVoxel=(9, 8, 7), dVoxel=(1.0, 1.1, 0.9), nDet=(13, 11), dDet=(0.83, 0.77), n=5, arc=math.pi):
    return inputs.parallel_geometry(nVoxel, dVoxel, nDet, dDet, n, arc=arc, DSO=60.0, DSD=100.0)


def brute_force_parallel(geo, vol, a, iu, iv):
    """delta * sum_k f(S_P + k delta r) over every k up to |D - S| / delta,
    f through the tent basis over all voxels; S_P = S + (P - D), r the unit
    central direction."""
    f = oracle.frames(geo)
    S, D = f["S"][a], f["D"][a]
    P = oracle.pixel_centres(geo, a)[iv, iu]
    SP = S + (P - D)
    L = np.linalg.norm(D - S)
    r = (D - S) / L
    delta = geo.accuracy * min(geo.dVoxel)
    n, d = np.asarray(geo.nVoxel), np.asarray(geo.dVoxel)
    h = 0.5 * n * d
    cs = [((np.arange(n[i]) + 0.5) - 0.5 * n[i]) * d[i] for i in range(3)]
    total = 0.0
    for k in range(int(math.floor(L / delta)) + 1):
        p = SP + k * delta * r
        if np.any(p < -h) or np.any(p > h):
            continue
        tx = np.maximum(0.0, 1.0 - np.abs(p[0] - cs[0]) / d[0])
        ty = np.maximum(0.0, 1.0 - np.abs(p[1] - cs[1]) / d[1])
        tz = np.maximum(0.0, 1.0 - np.abs(p[2] - cs[2]) / d[2])
        total += np.einsum("zyx,z,y,x->", vol, tz, ty, tx)
    return delta * total


def test_parallel_interp_matches_brute_force():
    g = _par(n=3)
    g.angles = np.stack([np.array([0.3, 1.9, 4.4]), np.array([0.0, 0.2, -0.1]), np.array([0.0, 0.1, 0.4])], axis=1)
    g.offDetector = np.array([[0.3, -0.2], [0.0, 0.5], [-0.4, 0.1]])
    g.accuracy = 0.37
    vol = np.random.default_rng(1).random(g.vol_shape)
    proj = oracle.forward(g, vol, "interp")
    for a in range(g.nAngles):
        for iv in range(g.nDetector[1]):
            for iu in range(g.nDetector[0]):
                assert proj[a, iv, iu] == pytest.approx(brute_force_parallel(g, vol, a, iu, iv), rel=1e-12,
                                                        abs=1e-12)


def test_parallel_gaussian_line_integrals():
    """Line integral s sqrt(2 pi) exp(-r^2 / (2 s^2)) along each parallel ray
    at distance r from the blob centre, within the trilinear-sampling bias
    bound of the cone-beam pin."""
    g = inputs.parallel_geometry((48, 48, 48), (1.0,) * 3, (40, 40), (1.0, 1.0), 4, arc=math.pi)
    g.accuracy = 0.25
    s, m = 6.0, np.array([2.0, -3.0, 1.5])
    c = [inputs.voxel_centres_1d(n, d) for n, d in zip(g.nVoxel, g.dVoxel)]
    X, Y, Z = c[0][None, None, :], c[1][None, :, None], c[2][:, None, None]
    vol = np.exp(-((X - m[0]) ** 2 + (Y - m[1]) ** 2 + (Z - m[2]) ** 2) / (2 * s * s))
    proj = oracle.forward(g, vol, "interp")
    f = oracle.frames(g)
    for a in range(g.nAngles):
        r = (f["D"][a] - f["S"][a]) / np.linalg.norm(f["D"][a] - f["S"][a])
        w = m - oracle.pixel_centres(g, a)
        r2 = np.sum(w * w, axis=-1) - (w @ r) ** 2
        ref = s * math.sqrt(2 * math.pi) * np.exp(-r2 / (2 * s * s))
        central = ref > 0.3 * ref.max()
        err = np.abs(proj[a] - ref)[central] / ref[central]
        assert err.max() < 1.3 / (4 * s * s)


def test_parallel_siddon_is_a_column_sum_at_angle_zero():
    """At angle 0 the rays run along -x at the pixel's (y, z): the Siddon
    line integral is dx times the sum of the column of voxels holding that
    (y, z)."""
    g = _par(n=1)
    vol = np.random.default_rng(2).random(g.vol_shape)
    proj = oracle.forward(g, vol, "siddon")[0]
    nu, nv = g.nDetector
    ny, nz = g.nVoxel[1], g.nVoxel[2]
    for iv in range(nv):
        for iu in range(nu):
            y = ((iu + 0.5) - 0.5 * nu) * g.dDetector[0]
            z = ((iv + 0.5) - 0.5 * nv) * g.dDetector[1]
            jy = math.floor(y / g.dVoxel[1] + 0.5 * ny)
            jz = math.floor(z / g.dVoxel[2] + 0.5 * nz)
            ref = g.dVoxel[0] * vol[jz, jy, :].sum() if 0 <= jy < ny and 0 <= jz < nz else 0.0
            assert proj[iv, iu] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_parallel_siddon_is_the_limit_of_a_distant_source():
    """A cone beam whose source is 1e7 mm away has rays within ~1e-6 rad of
    parallel: its Siddon projections agree with the parallel ones to ~1e-5."""
    g = _par(n=4)
    g.angles[:, 0] = [0.2, 1.1, 2.3, 3.0]
    far = inputs.circular_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, 4, 1.0e7, 1.0e7 + 40.0)
    far.angles = g.angles.copy()
    near = inputs.parallel_geometry(g.nVoxel, g.dVoxel, g.nDetector, g.dDetector, 4, DSO=1.0e7, DSD=1.0e7 + 40.0)
    near.angles = g.angles.copy()
    vol = np.random.default_rng(3).random(g.vol_shape)
    a = oracle.forward(far, vol, "siddon")
    b = oracle.forward(near, vol, "siddon")
    assert np.abs(a - b).max() < 1e-4 * np.abs(b).max()
    assert np.abs(a - b).max() > 0  # the two modes are different geometries


@pytest.mark.parametrize("method,bp", [("interp", "matched"), ("siddon", "siddon")])
def test_parallel_adjoint_identity(method, bp):
    g = _par(n=4)
    g.angles[:, 0] = [0.1, 0.9, 2.0, 2.8]
    g.rotDetector[:, 2] = 0.03
    rng = np.random.default_rng(4)
    x = rng.random(g.vol_shape)
    y = rng.random(g.proj_shape)
    lhs = np.sum(oracle.forward(g, x, method) * y)
    rhs = np.sum(x * oracle.backproject(g, y, bp))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_parallel_gather_form_equals_scatter():
    """Every voxel: the gather form (pixel search box from the parallel
    projection of the voxel's support) equals the scatter form."""
    g = _par(n=3)
    g.angles[:, 0] = [0.4, 1.7, 2.9]
    g.rotDetector[:, 0] = 0.05  # tilted detector: the rays are not along its normal
    g.rotDetector[:, 1] = 0.08
    y = np.random.default_rng(5).random(g.proj_shape)
    full = oracle.backproject(g, y, "matched")
    nx, ny, nz = g.nVoxel
    vox = np.array([[x, yy, z] for z in range(nz) for yy in range(ny) for x in range(nx)])
    got = oracle.backproject_voxels(g, y, vox, "matched")
    np.testing.assert_allclose(got, full.ravel(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("arc", [math.pi, 2 * math.pi])
@pytest.mark.parametrize("centre,R", [((0.0, 0.0), 15.0), ((7.0, -5.0), 9.0)])
def test_parallel_fbp_reconstructs_ball(arc, centre, R):
    """Parallel FBP (ramp at pitch du, no pre-weight, no distance weight,
    angle weight pi/nA) of the analytic projections 2 mu sqrt(R^2 - s^2) of
    a uniform ball, over a half or a full turn, returns mu inside the ball
    within 2 %.  The source plane sits 60 mm from the axis, so a leftover
    cone-beam distance weight (DSO/L)^2 would be off by several percent."""
    n = 90 if arc < 4 else 180
    g = inputs.parallel_geometry((48, 48, 16), (1.0,) * 3, (96, 20), (0.75, 1.0), n, arc=arc, DSO=60.0, DSD=100.0)
    mu = 0.02
    m = np.array([centre[0], centre[1], 0.0])
    f = oracle.frames(g)
    b = np.zeros(g.proj_shape)
    for a in range(g.nAngles):
        r = (f["D"][a] - f["S"][a]) / np.linalg.norm(f["D"][a] - f["S"][a])
        w = m - oracle.pixel_centres(g, a)
        s2 = np.sum(w * w, axis=-1) - (w @ r) ** 2
        b[a] = 2 * mu * np.sqrt(np.maximum(R * R - s2, 0.0))
    x = oracle.fdk(g, b)
    c = [inputs.voxel_centres_1d(nn, d) for nn, d in zip(g.nVoxel, g.dVoxel)]
    rr = np.sqrt((c[0][None, None, :] - m[0]) ** 2 + (c[1][None, :, None] - m[1]) ** 2 + 0 * c[2][:, None, None])
    inner = (rr < 0.6 * R) & (np.abs(c[2])[:, None, None] < 0.6 * R / 2)
    assert np.abs(x[inner] / mu - 1).max() < 0.02


def test_parallel_frequency_filter_equals_spatial_filter():
    """The windowed-filter path of the FDK variants reduces to the C
    oracle's spatial ramp on parallel scans too (no pre-weight, pitch du)."""
    from oracle import fdk_variants as ofdk
    g = _par(n=3)
    p = np.random.default_rng(6).standard_normal(g.proj_shape)
    a = ofdk.fdk_filter(g, p, "ram-lak")
    b = oracle.fdk_filter(g, p)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    with pytest.raises(ValueError):
        ofdk.fdk_filter(g, p, parker=True)
