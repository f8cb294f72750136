"""Pins of the oracle's geometry (Sec. 2.4, Appendix B parameter table)
against values derived by hand for the written convention."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def _geo(n_angles=4, **kw):
    g = inputs.circular_geometry((16, 16, 16), (1.0, 1.0, 1.0), (32, 24), (0.8, 0.6), n_angles, 1000.0, 1536.0)
    for k, v in kw.items():
        setattr(g, k, v)
    return g


def test_default_frame_by_hand():
    f = oracle.frames(_geo(1))
    np.testing.assert_allclose(f["S"][0], [1000.0, 0, 0], atol=1e-12)
    np.testing.assert_allclose(f["D"][0], [1000.0 - 1536.0, 0, 0], atol=1e-12)
    np.testing.assert_allclose(f["eu"][0], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(f["ev"][0], [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(f["n"][0], [-1, 0, 0], atol=1e-15)


def test_circular_orbit_rotates_source():
    g = _geo(8)
    f = oracle.frames(g)
    th = g.angles[:, 0]
    np.testing.assert_allclose(f["S"], np.stack([1000 * np.cos(th), 1000 * np.sin(th), 0 * th], 1), atol=1e-9)
    np.testing.assert_allclose(f["D"], np.stack([-536 * np.cos(th), -536 * np.sin(th), 0 * th], 1), atol=1e-9)
    # u axis follows the rotation of +y; v stays +z
    np.testing.assert_allclose(f["eu"], np.stack([-np.sin(th), np.cos(th), 0 * th], 1), atol=1e-12)
    np.testing.assert_allclose(f["ev"], np.tile([0, 0, 1.0], (8, 1)), atol=1e-12)


def test_offsets_by_hand():
    g = _geo(1)
    g.offOrigin = np.array([[3.0, -2.0, 5.0]])
    g.offDetector = np.array([[1.5, -0.5]])
    g.COR = np.array([0.7])
    f = oracle.frames(g)
    # origin shift moves source and detector the opposite way in volume frame
    np.testing.assert_allclose(f["S"][0], [1000 - 3.0, 0.7 + 2.0, -5.0], atol=1e-12)
    np.testing.assert_allclose(f["D"][0], [-536 - 3.0, 1.5 + 0.7 + 2.0, -0.5 - 5.0], atol=1e-12)


def test_zyz_angles_compose():
    g = _geo(1)
    z1, y1, z2 = 0.3, 0.2, -0.4
    g.angles = np.array([[z1, y1, z2]])
    f = oracle.frames(g)

    def Rz(a):
        return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])

    def Ry(a):
        return np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])

    R = Rz(z1) @ Ry(y1) @ Rz(z2)
    np.testing.assert_allclose(f["S"][0], R @ [1000, 0, 0], atol=1e-9)
    np.testing.assert_allclose(f["eu"][0], R @ [0, 1, 0], atol=1e-12)
    # a pure rotation keeps the detector frame orthonormal and right-handed
    M = np.stack([f["eu"][0], f["ev"][0], -f["n"][0]])
    np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-12)
    assert np.linalg.det(M) == pytest.approx(1.0)


def test_detector_in_plane_tilt():
    g = _geo(1)
    psi = 0.1
    g.rotDetector = np.array([[0.0, 0.0, psi]])
    f = oracle.frames(g)
    # rotation about the detector normal (x) turns u towards v
    np.testing.assert_allclose(f["eu"][0], [0, math.cos(psi), math.sin(psi)], atol=1e-12)
    np.testing.assert_allclose(f["ev"][0], [0, -math.sin(psi), math.cos(psi)], atol=1e-12)
    np.testing.assert_allclose(f["n"][0], [-1, 0, 0], atol=1e-12)


def test_central_ray_misses_centre_by_half_pixel():
    g = _geo(1)
    P = oracle.pixel_centres(g, 0)
    nu, nv = g.nDetector
    # pixel (nu/2, nv/2) is the first one above/right of the detector centre
    np.testing.assert_allclose(P[nv // 2, nu // 2], [-536, 0.4, 0.3], atol=1e-12)
    np.testing.assert_allclose(P[0, 0], [-536, -(nu / 2 - 0.5) * 0.8, -(nv / 2 - 0.5) * 0.6], atol=1e-12)


def _ball(geo, centre, radius, mu=1.0):
    nx, ny, nz = geo.nVoxel
    c = [inputs.voxel_centres_1d(n, d) for n, d in zip(geo.nVoxel, geo.dVoxel)]
    X, Y, Z = c[0][None, None, :], c[1][None, :, None], c[2][:, None, None]
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    return (r2 <= radius * radius).astype(np.float64) * mu


def test_centred_ball_projects_symmetrically():
    g = inputs.circular_geometry((24, 24, 24), (1.0,) * 3, (40, 30), (0.9, 0.9), 3, 1000.0, 1536.0)
    vol = _ball(g, (0, 0, 0), 8.0)
    for method in ("siddon", "interp"):
        p = oracle.forward(g, vol, method)[0]
        np.testing.assert_allclose(p, p[:, ::-1], rtol=0, atol=1e-10 * p.max())
        np.testing.assert_allclose(p, p[::-1, :], rtol=0, atol=1e-10 * p.max())


@pytest.mark.parametrize("theta,expected_u", [
    (0.0, 10.0 * 1536 / 1000),          # ball towards +u
    (math.pi, -10.0 * 1536 / 1000),     # u axis flipped
    (math.pi / 2, 0.0),                 # ball on the central ray
])
def test_offcentre_ball_shadow_moves_as_predicted(theta, expected_u):
    g = inputs.circular_geometry((48, 48, 16), (0.5,) * 3, (1024, 32), (0.05, 0.2), 1, 1000.0, 1536.0,
                                 start=theta)
    vol = _ball(g, (0.0, 10.0, 0.0), 1.5)
    p = oracle.forward(g, vol, "siddon")[0].sum(axis=0)
    u = ((np.arange(1024) + 0.5) - 512) * 0.05
    centroid = float((p * u).sum() / p.sum())
    # perspective moves the centroid of a ball's shadow by ~1e-5 relative;
    # the pixel quadrature of the shadow profile by ~(du)^2
    assert centroid == pytest.approx(expected_u, abs=0.005)


@pytest.mark.parametrize("axis", ["phi", "theta"])
def test_detector_rotation_single_axes(axis):
    g = _geo(1)
    a = 0.2
    g.rotDetector = np.array([[a, 0.0, 0.0]] if axis == "phi" else [[0.0, a, 0.0]])
    f = oracle.frames(g)
    if axis == "phi":   # about z: u turns towards -x, v stays
        np.testing.assert_allclose(f["eu"][0], [-math.sin(a), math.cos(a), 0], atol=1e-12)
        np.testing.assert_allclose(f["ev"][0], [0, 0, 1], atol=1e-12)
        np.testing.assert_allclose(f["n"][0], [-math.cos(a), -math.sin(a), 0], atol=1e-12)
    else:               # about y: v turns towards +x, u stays
        np.testing.assert_allclose(f["eu"][0], [0, 1, 0], atol=1e-12)
        np.testing.assert_allclose(f["ev"][0], [math.sin(a), 0, math.cos(a)], atol=1e-12)
    # the detector rotates about its own centre D
    np.testing.assert_allclose(f["D"][0], [-536.0, 0, 0], atol=1e-12)
