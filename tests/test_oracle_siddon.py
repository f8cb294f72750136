"""Pins of the oracle's Siddon projector: b_i = sum_j x_j |segment_i & cell_j|
(Eq. 1 with exact intersection lengths) against closed-form chord lengths
computed per cell by the slab method, independently of the merged-crossing
walk the oracle uses."""
import numpy as np
import pytest

import oracle
from paper_2412_10129_gb300 import inputs


def slab_length(S, P, lo, hi):
    """Length of the segment S->P inside the box [lo, hi] (closed form)."""
    d = P - S
    t0, t1 = 0.0, 1.0
    for a in range(3):
        if d[a] == 0.0:
            if S[a] < lo[a] or S[a] > hi[a]:
                return 0.0
            continue
        ta, tb = (lo[a] - S[a]) / d[a], (hi[a] - S[a]) / d[a]
        ta, tb = min(ta, tb), max(ta, tb)
        t0, t1 = max(t0, ta), min(t1, tb)
    return max(0.0, t1 - t0) * float(np.linalg.norm(d))


def _rays(g):
    f = oracle.frames(g)
    for a in range(g.nAngles):
        P = oracle.pixel_centres(g, a)
        for iv in range(g.nDetector[1]):
            for iu in range(g.nDetector[0]):
                yield a, iv, iu, f["S"][a], P[iv, iu]


def test_siddon_constant_volume_is_box_chord():
    g = inputs.random_geometry((7, 6, 5), (1.0, 1.2, 0.9), (11, 9), (1.2, 1.1), 3, seed=4, DSO=60.0, DSD=110.0)
    proj = oracle.forward(g, np.ones(g.vol_shape), "siddon")
    h = 0.5 * np.asarray(g.nVoxel) * np.asarray(g.dVoxel)
    for a, iv, iu, S, P in _rays(g):
        assert proj[a, iv, iu] == pytest.approx(slab_length(S, P, -h, h), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_siddon_random_volume_equals_per_cell_chords(seed):
    g = inputs.random_geometry((5, 4, 4), (1.0, 1.1, 0.9), (8, 7), (1.0, 1.0), 2, seed=seed, DSO=50.0, DSD=90.0)
    vol = np.random.default_rng(seed).random(g.vol_shape)
    proj = oracle.forward(g, vol, "siddon")
    n, d = np.asarray(g.nVoxel), np.asarray(g.dVoxel)
    for a, iv, iu, S, P in _rays(g):
        ref = 0.0
        for iz in range(n[2]):
            for iy in range(n[1]):
                for ix in range(n[0]):
                    lo = (np.array([ix, iy, iz]) - 0.5 * n) * d
                    ref += vol[iz, iy, ix] * slab_length(S, P, lo, lo + d)
        assert proj[a, iv, iu] == pytest.approx(ref, rel=1e-11, abs=1e-12)


def test_siddon_axis_aligned_ray():
    """A ray along x through the interior crosses n_x cells of width d_x."""
    g = inputs.circular_geometry((6, 5, 5), (1.5, 1.0, 1.0), (3, 3), (1.0, 1.0), 1, 100.0, 200.0)
    vol = np.random.default_rng(0).random(g.vol_shape)
    # pixel (1, 1) of a 3x3 detector is on the central ray: y = z = 0 lies on
    # the mid-plane between cells for even counts; use odd counts (5) here.
    proj = oracle.forward(g, vol, "siddon")
    assert proj[0, 1, 1] == pytest.approx(1.5 * vol[2, 2, :].sum(), rel=1e-13)


def test_siddon_adjoint_identity():
    g = inputs.random_geometry((8, 7, 6), (1.0, 1.0, 1.1), (12, 10), (1.1, 1.2), 4, seed=3, DSO=80.0, DSD=140.0)
    rng = np.random.default_rng(1)
    x, y = rng.random(g.vol_shape), rng.random(g.proj_shape)
    lhs = float(np.sum(oracle.forward(g, x, "siddon") * y))
    rhs = float(np.sum(x * oracle.backproject(g, y, "siddon")))
    assert abs(lhs - rhs) / lhs < 1e-12
